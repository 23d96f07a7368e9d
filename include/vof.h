/*
 * gvof: GB300 (sm_103a) CUDA library for the data-parallel hot path of the
 * unsplit geometric volume-of-fluid method of arXiv 2111.01524 (gVOF):
 * LSGIR reconstruction (Sec. 2.1.1), optionally refined by LSFIR (Sec.
 * 2.1.2), with a volume-enforcing plane constant (Sec. 2.1); FMFPA
 * face-matched (Sec. 2.2.2), EMFPA edge-matched (Sec. 2.2.1) or NMFPA
 * non-matched (Sec. 2.2.3) flux polyhedra truncated by the upstream cells'
 * PLIC half-spaces (Sec. 2.2); and the conservative update of Eq. fnext with
 * the final clip (Sec. 2.2).
 *
 * Conventions
 *  - Mesh: OpenFOAM-like face-based polyhedral mesh (Sec. 3.1). Faces are
 *    planar polygons; their nodes run counter-clockwise seen from outside
 *    the owner cell, so the right-hand normal leaves the owner. A boundary
 *    face has neighbour = -1. Cells may be convex or non-convex (e.g. the
 *    distorted cubic cells with triangulated faces of Sec. 4); a cell has
 *    at most 32 faces, 32 nodes and 128 face-node entries.
 *  - PLIC plane of an interfacial cell (Eq. plic-eq):  n.(x - xc) + C = 0,
 *    xc = cell centroid, n = unit normal pointing into the fluid; the fluid
 *    is the part of the cell where n.(x - xc) + C >= 0.
 *  - Face volumes V_d (Eq. a-donacion) and V_F are positive when they leave
 *    the owner cell.
 *  - Tags (Sec. 3.3): -1 / 0 / 1 for empty / interfacial / full.
 *  - Every function returns a vof_status; on failure vof_last_error() gives
 *    a message (thread-local). No function aborts or traps the GPU.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Device work
 *    is queued on it. A function given HOST buffers synchronises the stream
 *    before returning; one given DEVICE buffers does not.
 *  - Ownership: the caller owns every buffer it passes; the library copies
 *    what it keeps. The context owns all device memory it allocates and
 *    frees it in vof_destroy.
 */
#ifndef GVOF_VOF_H
#define GVOF_VOF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VOF_OK = 0,
  VOF_EINVAL = 1,    /* invalid argument or mesh */
  VOF_ENOMEM = 2,    /* device or host allocation failed */
  VOF_ECUDA = 3,     /* a CUDA call failed */
  VOF_ECAPACITY = 4, /* a fixed-capacity buffer overflowed (see stats) */
  VOF_ESTATE = 5,    /* call out of order (e.g. advect before reconstruct) */
  VOF_ECFL = 6       /* flux polyhedra left their candidate cells (see vof_get_stats) */
} vof_status;

enum { VOF_PREC_FP64 = 0, VOF_PREC_MIXED = 1 };
enum { VOF_MEM_HOST = 0, VOF_MEM_DEVICE = 1 };
enum { VOF_VEL_DEFORMATION = 1, VOF_VEL_ROTATION = 2, VOF_VEL_TRANSLATION = 3,
       VOF_VEL_DEFORMATION2D = 4 };
/* flux polyhedron construction (vof_options.flux_polyhedron) */
enum { VOF_FLUX_FMFPA = 0, VOF_FLUX_EMFPA = 1, VOF_FLUX_NMFPA = 2 };
/* interface reconstruction (vof_options.reconstruction) */
enum { VOF_RECON_LSGIR = 0, VOF_RECON_LSFIR = 1 };
/* points per face in vof_get_flux_polyhedra: 3I+1 for an EMFPA face of
 * I <= 6 nodes, 2I+1 for an FMFPA face of I <= 8 */
enum { VOF_MAX_POLY_VERTS = 19 };

typedef struct vof_ctx vof_ctx;

/* Face-based mesh (Sec. 3.1), HOST arrays, read during vof_init only.
 * X: [3*n_vert] interleaved x,y,z. face_ptr: [n_face+1] CSR offsets into
 * face_vert (3..8 nodes per face). owner, neighbour: [n_face]. */
typedef struct {
  int64_t n_vert, n_face, n_cell;
  const double* X;
  const int64_t* face_ptr;
  const int32_t* face_vert;
  const int32_t* owner;
  const int32_t* neighbour;
} vof_mesh_desc;

/* eps: volume-fraction tolerance of Sec. 2.1 and Sec. 3.3 (paper: 1e-12).
 * beta: LSGIR weight exponent of Eq. lsgir-beta (paper: 1.5).
 * precision: VOF_PREC_FP64 (all geometry in FP64) or VOF_PREC_MIXED
 * (geometry in FP32 in face- or cell-local scaled coordinates; FP64 for the
 * plane constant of cells with F or 1-F below 1e-3, for V_d, for the
 * per-face flux sums, the cell update and global sums).
 * flux_polyhedron: VOF_FLUX_FMFPA (Sec. 2.2.2: 2I+1 faces, side faces
 * parallel to the edge-centre velocity) or VOF_FLUX_EMFPA (Sec. 2.2.1:
 * 5I+1 faces, each vertex back-traced with its own velocity, side faces
 * split into four triangles) or VOF_FLUX_NMFPA (Sec. 2.2.3: I+2 planar
 * faces, every vertex moved back with the face-centre velocity; not
 * strictly conservative, as the paper notes). EMFPA needs every face to
 * have at most 6 nodes (its 31 faces fill the per-face capacity); vof_init
 * returns VOF_EINVAL otherwise.
 * reconstruction: VOF_RECON_LSGIR (Sec. 2.1.1) or VOF_RECON_LSFIR (Sec.
 * 2.1.2: from the LSGIR planes, up to lsfir_max_iter outer iterations, each
 * fitting every interfacial cell's normal to the PLIC vertex-average
 * centres of its valid neighbours (weights |dx|^-2.5, previous normals
 * within 45 degrees), taking it where it turns the normal by less than
 * 30 degrees / iteration, and enforcing the plane constants again; stops
 * after an iteration in which no accepted turn reached lsfir_tol radians).
 * lsfir_max_iter: 0 means 4 (the paper's n_out), at most 16. lsfir_tol: 0
 * means 1e-3 rad.
 * poly_capacity: how many active faces per step get their flux polyhedron
 * built ahead of the flux kernel (one thread per face) into a buffer of
 * (3 * 19 + 7) values per face in the path's precision; active faces beyond
 * it are built inside the flux kernel by one lane, with the same arithmetic,
 * so results do not depend on it. 0 means min(n_face, 4 Mi); otherwise
 * 1..n_face (VOF_EINVAL if negative). A GPU memory/latency trade-off with no
 * counterpart in the paper.
 * faces_per_warp: flux polyhedra truncated by one warp: 1, or 2 (each face
 * by half a warp, 16 lanes, which holds at most 16 face loops; allowed for
 * FMFPA and NMFPA on grids whose cells are all convex and where the
 * polyhedron's faces (3I+1 for FMFPA, I+2 for NMFPA, I the most nodes of a
 * face) plus the most faces of a cell plus one number at most 16, e.g.
 * FMFPA on tetrahedra and NMFPA on hexahedra; VOF_EINVAL otherwise), or 0
 * for the library's choice (1). Every reduction keeps its order, so the
 * results are the same bit for bit either way. vof_autotune_ex
 * may change it. */
typedef struct {
  double eps;
  double beta;
  int32_t precision;
  int32_t flux_polyhedron;
  int32_t reconstruction;
  int32_t lsfir_max_iter;
  double lsfir_tol;
  int32_t poly_capacity;
  int32_t faces_per_warp;
} vof_options;

/* Prescribed velocity of the test problems (Sec. 4.2, Sec. 4.3):
 * DEFORMATION: Enright field of Sec. 4.2.3 with period `period`;
 * DEFORMATION2D: the x-z field of the 2D deformation test (Sec. 4.3),
 *   u = -2 sin^2(pi x) sin(pi z) cos(pi z) g, v = 0,
 *   w = 2 sin^2(pi z) sin(pi x) cos(pi x) g, g = cos(pi t / period);
 * ROTATION: u = -omega (y - center[1]), v = omega (x - center[0]), w = 0;
 * TRANSLATION: u = u0. Velocities are evaluated exactly at face centres,
 * edge centres and vertices at the mid-time t + dt/2 (Sec. 4.2). */
typedef struct {
  int32_t kind;
  int32_t pad;
  double period;
  double omega;
  double center[3];
  double u0[3];
} vof_velocity;

/* Counters and sums of the last advect / reconstruct (vof_get_stats). */
typedef struct {
  int64_t n_interfacial;  /* cells with tag 0 */
  int64_t n_active_faces; /* faces with tag 0 (geometric flux) */
  int64_t n_truncations;  /* (face, cell) truncations evaluated */
  int64_t n_overflow;     /* polyhedra that overflowed a buffer: their V_F is unreliable */
  int64_t n_degenerate;   /* FMFPA side lines replaced by the streak-line point */
  int64_t n_edgeon;       /* FMFPA faces whose back-traced loop was edge-on */
  double volume;          /* sum over cells of V F (FP64, fixed-order) */
  double ebound;          /* E_bound^Linf of Sec. 4.2 before the clip of the last advect */
  /* Volume bookkeeping since the last vof_set_fraction (Sec. 2.2, Eq. fnext
   * and the final clip; Sec. 2.1 cut-off), each summed in a fixed order:
   * volume == V_0 - clip_loss - cutoff_loss - boundary_outflow, V_0 the
   * volume of the F that was set, up to rounding (the update conserves the
   * fluid that the face volumes move; only these three terms change it). */
  double clip_loss;         /* sum over cells and steps of V (F_unclipped - F) */
  double cutoff_loss;       /* sum of V (F - F_cut) removed by the cut-off to 0 / 1 */
  double boundary_outflow;  /* sum of V_F over boundary faces (fluid leaving the domain) */
  /* last advect: */
  int64_t n_clipped;   /* cells whose Eq. fnext value left [0, 1] and was clipped */
  int64_t n_repaired;  /* mixed path: face volumes adjusted to hand FP32 noise back
                        * to neighbours with room (see vof_advect) */
  int64_t n_escaped;   /* flux polyhedra with a vertex inside the domain but outside
                        * every candidate cell (CFL too large for the candidate
                        * ring; their V_F misses that part): vof_get_stats then
                        * returns VOF_ECFL */
} vof_stats;

/* Create a context: copies the mesh to the device and builds its derived
 * connectivity (neigbcell, cell->face, cell->vertex, vertex->cell) and
 * geometry (compgrid), Sec. 3.1. opt may be NULL (defaults). The copies and
 * geometry kernels run on `stream`, which is synchronised before return
 * (the mesh arrays may be freed then). */
vof_status vof_init(const vof_mesh_desc* mesh, const vof_options* opt, void* stream,
                    vof_ctx** out);
void vof_destroy(vof_ctx* ctx);
const char* vof_last_error(void);

/* Batching: n_grids independent meshes joined into one context. Cells,
 * faces and nodes of grid g follow those of grid g-1 (offsets from
 * vof_batch_offsets), so every kernel of a step processes all grids in one
 * launch; each grid keeps its own velocity field and time step (the
 * *_batch calls take arrays of n_grids velocities, times and steps). A
 * context made by vof_init is a batch of one grid. */
vof_status vof_batch_create(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                            void* stream, vof_ctx** out);
/* vof_batch_create on the legacy default stream */
vof_status vof_init_batch(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                          vof_ctx** out);
/* offsets [n_grids+1] of each grid's cells, faces, nodes (any may be NULL) */
vof_status vof_batch_offsets(vof_ctx* ctx, int* n_grids, int64_t* cell_off, int64_t* face_off,
                             int64_t* vert_off);

/* Initial fluid body for vof_init_fraction (initfgrid, Sec. 3.2): the fluid
 * is where the body's signed distance is negative.
 * VOF_SHAPE_SPHERE: centre c, radius r. VOF_SHAPE_CYLINDER: infinite, axis
 * through c along the unit vector a, radius r. VOF_SHAPE_HALFSPACE:
 * a.(x - c) < 0 with a a unit vector (r unused). */
enum { VOF_SHAPE_SPHERE = 1, VOF_SHAPE_CYLINDER = 2, VOF_SHAPE_HALFSPACE = 3 };
typedef struct {
  int32_t kind;
  int32_t pad;
  double c[3];
  double a[3];
  double r;
} vof_shape;

/* initfgrid (Sec. 3.2) on the device: F of every cell by refinement. Each
 * cell is the signed sum of the tetrahedra joining its vertex average to
 * the fan triangles (face vertex average, edge) of its faces; each
 * tetrahedron is divided into ndiv^3 equal tetrahedra (Freudenthal) on
 * which the fluid is where the linear interpolant of the signed distance
 * is negative. Cells whose bounding ball about the centroid lies on one
 * side of the surface get 0 or 1. ndiv in 1..16 (the paper uses 10). Every
 * grid of a batch gets the same body. Replaces F like vof_set_fraction
 * (the reconstruction must follow); asynchronous on `stream`.
 * VOF_EINVAL for an unknown kind, a non-unit axis or normal (|1 - |a|| >
 * 1e-12), r <= 0 for a sphere or cylinder, or ndiv out of range. */
vof_status vof_init_fraction(vof_ctx* ctx, const vof_shape* shape, int ndiv, void* stream);

/* Volume fraction F [n_cell] (host or device pointer, see `mem`). Setting F
 * invalidates the reconstruction: call vof_reconstruct next. The volume
 * bookkeeping of vof_stats restarts from this F. When F differs from the
 * library's copy only in cells the last advect could change (its band:
 * owner and neighbour of each active face, and the interfacial cells), the
 * next sweeps stay band-limited, so a caller that reads F back and sets it
 * again each step pays no full sweep; any other change makes them full. The
 * results are those of full sweeps either way. A host F goes through a
 * device copy and the call synchronises the stream before it returns.
 * VOF_EINVAL for a NULL argument or (host F) a mesh with fewer faces than
 * cells, which no closed mesh has. */
vof_status vof_set_fraction(vof_ctx* ctx, const double* F, int mem, void* stream);
vof_status vof_get_fraction(vof_ctx* ctx, double* F, int mem, void* stream);

/* taggrid (cut-off of F, node F* by inverse-distance weighting, node/face/
 * cell tags; Sec. 2.1, Sec. 3.3) then LSGIR normals and plane constants of
 * the interfacial cells (Secs. 2.1, 2.1.1), refined by the LSFIR outer
 * iteration (Sec. 2.1.2) when the context was made with
 * VOF_RECON_LSFIR. */
vof_status vof_reconstruct(vof_ctx* ctx, void* stream);

/* faceflux + vofadv (Sec. 3.5): V_d of every face (Eq. a-donacion), FMFPA
 * flux polyhedra of the tag-0 faces truncated by the PLIC half-spaces of
 * the overlapped cells (Sec. 2.2), V_F = 0 / V_d on tag -1 / 1 faces, then
 * Eq. fnext and the clip to [0, 1]. Velocity at t + dt/2. Requires a
 * reconstruction of the current F.
 * Mixed precision: the face volumes of truncated polyhedra carry FP32
 * rounding (a few ulps of A^(3/2) per face, A its area), which can push a
 * nearly full or empty cell past [0, 1] where the clip would turn it into
 * lost volume. A cell whose Eq. fnext value leaves [0, 1] by more than 1e-14
 * and by no more than that noise (2e-6 times the sum of A^(3/2) over its
 * inexact faces, and 5e-7 of its own volume) is not clipped at once: the
 * excess goes back through its inexact faces to the neighbours with room
 * (space for an overfull cell, fluid for an overdrawn one), in proportion
 * to that room, each adjustment one face volume applied with opposite
 * signs to its two cells; Eq. fnext is applied again from the F before the
 * step to the cells of the adjusted faces (three rounds; the last clips
 * every cell, the paper's clip). A larger excess is the method's own and is
 * clipped as in the FP64 path. The global volume then follows the FP64
 * path's (tested to 1e-12 relative on hexahedral grids). */
vof_status vof_advect(vof_ctx* ctx, const vof_velocity* vel, double t, double dt, void* stream);
/* the same call under the name of the method's step (Algorithm alg:adv) */
vof_status vof_advect_step(vof_ctx* ctx, const vof_velocity* vel, double t, double dt,
                           void* stream);

/* One iteration of the advection test loop (Algorithm alg:adv):
 * vof_advect followed by vof_reconstruct. */
vof_status vof_step(vof_ctx* ctx, const vof_velocity* vel, double t, double dt, void* stream);

/* Time step of Eq. eq:cfl at time t: CFL times the smallest ratio, over the
 * axes, of the smallest cell bounding-box size to the largest face-centre
 * speed; refined once with the field at t + dt and cut to reach t_end.
 * Host result; the first call for a velocity field runs a device sweep. */
vof_status vof_suggest_dt(vof_ctx* ctx, const vof_velocity* vel, double t, double cfl,
                          double t_end, double* dt);

/* Batched forms: vels, t, dt, t_end, dt_out are HOST arrays of n_grids. */
vof_status vof_advect_batch(vof_ctx* ctx, const vof_velocity* vels, const double* t,
                            const double* dt, void* stream);
vof_status vof_step_batch(vof_ctx* ctx, const vof_velocity* vels, const double* t,
                          const double* dt, void* stream);
/* vof_step_batch under its batch name */
vof_status vof_batch_step(vof_ctx* ctx, const vof_velocity* vels, const double* t,
                          const double* dt, void* stream);
vof_status vof_suggest_dt_batch(vof_ctx* ctx, const vof_velocity* vels, const double* t,
                                double cfl, const double* t_end, double* dt_out);

/* ---- Partitioned grids (domain decomposition) ----------------------------
 * One grid split into parts, each part a context of its own on the part's
 * cells plus a halo of node-neighbour rings (a sub-mesh, cells and faces in
 * the grid's order); every step each part advects, the halo cells receive
 * F of their owning parts, and each part reconstructs. With a halo deep
 * enough for the step's stencils (Secs. 2.1, 2.2, 3.5: the donating-region
 * candidates of a face are the node neighbours of its two cells, and a
 * plane reads F of its cell's node neighbours), the owned cells' F equals
 * the unpartitioned grid's bit for bit.
 *
 * vof_halo_lists: the context's cell lists (HOST arrays): list k is
 * cells[ptr[k] .. ptr[k+1]-1], cell indices of this context (any order,
 * repeats allowed); ptr has n_lists + 1 entries, ptr[0] = 0, non-decreasing.
 * Copied to the device (the context owns the copy; earlier lists are
 * replaced; waits for the device). VOF_EINVAL for a bad ptr or an index
 * outside 0..n_cell-1. */
vof_status vof_halo_lists(vof_ctx* ctx, int n_lists, const int64_t* ptr, const int32_t* cells);
/* out[i] = F[cells[i]] over list `list` (out: DEVICE, list size doubles),
 * asynchronous on `stream` */
vof_status vof_halo_export(vof_ctx* ctx, int list, double* out, void* stream);
/* F[cells[i]] = in[i] over list `list` (in: DEVICE), asynchronous on
 * `stream`; like vof_set_fraction the next advect needs a vof_reconstruct,
 * and the next sweeps stay band-limited only if every changed cell was in
 * the band of the last advect */
vof_status vof_halo_import(vof_ctx* ctx, int list, const double* in, void* stream);
/* *vol = sum of V_k F_k over the cells of list `list`, in a fixed order
 * (HOST result; synchronises `stream`) */
vof_status vof_list_volume(vof_ctx* ctx, int list, double* vol, void* stream);
/* The bounds Eq. eq:cfl takes over a grid: per axis the smallest cell
 * bounding-box size and the largest face-centre speed of the velocity
 * field's spatial part (HOST double[3] each; single-grid contexts). The
 * bounds of a partitioned grid are the minimum and maximum over its parts,
 * and vof_dt_from_bounds turns them into vof_suggest_dt's time step: the
 * same value, bit for bit, as the unpartitioned grid's. */
vof_status vof_dt_bounds(vof_ctx* ctx, const vof_velocity* vel, double* hmin, double* umax);
vof_status vof_dt_from_bounds(const vof_velocity* vel, const double* hmin, const double* umax,
                              double t, double cfl, double t_end, double* dt);

/* CUDA graph of one step: vof_graph_capture records the launches of one
 * vof_advect (with_reconstruct = 0) or vof_step (1) on `stream` (not the
 * legacy default stream) into a graph; vof_graph_launch writes the step's
 * per-grid parameters into device memory (an asynchronous copy from a pinned
 * ring) and replays the graph. The kernels read every per-step value from
 * that device table, so one graph serves all steps. Re-capture after
 * vof_autotune. */
vof_status vof_graph_capture(vof_ctx* ctx, int with_reconstruct, void* stream);
vof_status vof_graph_launch(vof_ctx* ctx, const vof_velocity* vels, const double* t,
                            const double* dt, void* stream);

/* Launch-shape autotuner: times the flux and reconstruction kernels on the
 * current state and keeps the fastest: blocks per SM of each (2..16), faces
 * per warp of the flux kernel (1, and 2 where vof_options.faces_per_warp
 * allows it) and whether the flux polyhedra are prebuilt into the
 * poly_capacity buffer ahead of the flux kernel or built inside it. The
 * choices are returned through the pointers that are not NULL
 * (prebuilt: 1 or 0). Results do not depend on any of them. F and the
 * reconstruction are left unchanged; the face volumes are those of a step
 * (t, dt). Re-capture a graph after it. */
vof_status vof_autotune(vof_ctx* ctx, const vof_velocity* vels, const double* t, const double* dt,
                        void* stream, int* flux_blocks, int* recon_blocks);
vof_status vof_autotune_ex(vof_ctx* ctx, const vof_velocity* vels, const double* t,
                           const double* dt, void* stream, int* flux_blocks, int* recon_blocks,
                           int* faces_per_warp, int* prebuilt);

/* planes [4*n_cell]: nx, ny, nz, C per cell (zeros for non-interfacial). */
vof_status vof_get_planes(vof_ctx* ctx, double* planes, int mem, void* stream);
/* tags: any pointer may be NULL; sizes n_vert, n_face, n_cell. */
vof_status vof_get_tags(vof_ctx* ctx, int8_t* tag_v, int8_t* tag_f, int8_t* tag_c, int mem,
                        void* stream);
/* face volumes of the last advect [n_face]; either pointer may be NULL. */
vof_status vof_get_face_flux(vof_ctx* ctx, double* Vd, double* VF, int mem, void* stream);
/* compgrid geometry: cell_vol [n_cell], cell_cen [3*n_cell], face_cen
 * [3*n_face], face_nrm [3*n_face], face_area [n_face]; any may be NULL. */
vof_status vof_get_geometry(vof_ctx* ctx, double* cell_vol, double* cell_cen, double* face_cen,
                            double* face_nrm, double* face_area, int mem, void* stream);
/* neigbcell CSR (cells sharing >= 1 node, self excluded, ascending), HOST
 * buffers: ptr [n_cell+1]; idx [*count]. Pass idx = NULL to query count. */
vof_status vof_get_neighbors(vof_ctx* ctx, int64_t* ptr, int32_t* idx, int64_t* count);
/* Overlap candidates of faces, computed by the same device routine the flux
 * kernel uses: owner, neighbour and their node neighbours, ascending.
 * faces: HOST [n]; out_ptr HOST [n+1]; out_idx HOST [cap]. */
vof_status vof_get_candidates(vof_ctx* ctx, const int32_t* faces, int n, int64_t* out_ptr,
                              int32_t* out_idx, int64_t cap);
/* Flux polyhedra of the given faces built by the device routine the flux
 * kernel uses, with the context's construction: verts HOST [n *
 * VOF_MAX_POLY_VERTS * 3] absolute coordinates, padded with zeros; FMFPA
 * (Sec. 2.2.2): 2I+1 points per face (x_1..x_I, back-traced x_{I+1}..x_{2I},
 * apex); EMFPA (Sec. 2.2.1): 3I+1 points (x_1..x_I, back-traced
 * x_{I+1}..x_{2I}, side-face centres s_1..s_I, apex); NMFPA (Sec. 2.2.3):
 * 2I points (x_1..x_I, x_i - dt u_c). counts HOST [n] receives I. */
vof_status vof_get_flux_polyhedra(vof_ctx* ctx, const vof_velocity* vel, double t, double dt,
                                  const int32_t* faces, int n, double* verts, int32_t* counts);
/* Checkpoint / resume (no counterpart in the paper): the state a step
 * continues from, taken after a reconstruction (vof_reconstruct or
 * vof_step): F, the PLIC planes (n, C) and the node and cell tags of the last
 * reconstruction, and the volume bookkeeping. buf is an opaque HOST buffer
 * of *need bytes (vof_get_state with buf = NULL only reports *need). A
 * context of the same mesh (cell and node counts are checked) restored with
 * vof_set_state continues like the one that saved it: F and the planes bit
 * for bit (its next sweeps are full, which give the band-limited sweeps'
 * results), the bookkeeping sums to rounding (their per-block partial sums
 * follow the sweep's assignment of cells to blocks). Both
 * synchronise `stream`. VOF_ESTATE if the reconstruction is not current;
 * VOF_EINVAL for a short or foreign buffer. */
vof_status vof_get_state(vof_ctx* ctx, void* buf, int64_t bytes, int64_t* need, void* stream);
vof_status vof_set_state(vof_ctx* ctx, const void* buf, int64_t bytes, void* stream);

/* counters and global sums (synchronises the stream). Returns VOF_ECFL,
 * with *out filled in, when flux polyhedra of the last advect reached past
 * their candidate cells (n_escaped > 0, Sec. 2.2 with the CFL condition of
 * Sec. 3.3): their V_F misses the part outside the cells around the face;
 * a smaller time step (Eq. eq:cfl with a smaller CFL number) avoids it. */
vof_status vof_get_stats(vof_ctx* ctx, vof_stats* out, void* stream);
/* Per-phase device timing with CUDA events recorded on the launching
 * stream around each kernel of the step (off by default). Phases:
 * 0 cell tags, 1 node tags, 2 reconstruct (LSGIR or LSFIR + plane
 * constant), 3 face sweep, 4 flux (truncation of the flux polyhedra),
 * 5 update, 6 polyhedra (their construction, Sec. 2.2), 7 repair (mixed
 * precision: FP64 face volumes of cells the clip would cut). vof_get_timing
 * synchronises, returns the accumulated milliseconds and kernel launch
 * counts (band-list kernels included) of the first n phases and resets
 * them. */
enum { VOF_PHASE_CELL_TAGS = 0, VOF_PHASE_NODE_TAGS = 1, VOF_PHASE_RECONSTRUCT = 2,
       VOF_PHASE_FACE_SWEEP = 3, VOF_PHASE_FLUX = 4, VOF_PHASE_UPDATE = 5,
       VOF_PHASE_POLYHEDRA = 6, VOF_PHASE_REPAIR = 7, VOF_NUM_PHASES = 8 };
vof_status vof_set_timing(vof_ctx* ctx, int on);
vof_status vof_get_timing(vof_ctx* ctx, double* ms, int64_t* launches, int n);
/* Allocation-free weighted sum: *out = sum over i < n of w[i] * F[i] (the
 * global fluid volume when w holds the cell volumes), in the same fixed
 * order on every call. The paper has no counterpart; this entry point
 * exists for callers that cannot allocate device memory where they need the
 * sum, e.g. a solver that reserved its whole device budget up front, or a
 * time loop that must not pay the device-wide synchronisation or the
 * failure modes of cudaMalloc. w, F and out are DEVICE pointers owned by the
 * caller; the result is written to out[0] asynchronously on `stream`.
 * It allocates nothing: its only scratch is a file-scope device array of
 * 65536 doubles (512 KiB) that every GPU loading the library holds until
 * the process exits, so n is limited to 65536 * 4096 = 268,435,456;
 * larger (or negative) n returns VOF_EINVAL with a message. The first call
 * on a device looks up that array's device address (set-up, once per
 * device); make that first call before any stream capture. All calls share
 * the array: calls that overlap on the GPU (different streams, or different
 * host threads using one device) race, so serialise them. */
vof_status vof_volume_sum_noalloc(const double* w, const double* F, int64_t n, double* out,
                                  void* stream);
/* bytes of device memory held by the context */
int64_t vof_device_bytes(const vof_ctx* ctx);
/* bytes of device memory that vof_batch_create(meshes, n_grids, opt) would
 * allocate (equal to the new context's vof_device_bytes), computed on the
 * host from the mesh sizes and their derived connectivity; opt may be NULL
 * (defaults). No GPU work. VOF_EINVAL for an invalid mesh. */
vof_status vof_estimate_bytes(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                              int64_t* bytes);

/* Serving (continuous batching of "advance this interface N steps"
 * requests; no counterpart in the paper, whose tests are single runs).
 * A request is a mesh, its initial F, a velocity field of Sec. 4.2/4.3, a
 * number of steps, a CFL number and an end time (Eq. eq:cfl gives each
 * step). vof_server_step is one scheduling tick: it collects the results of
 * requests whose last step completed, admits queued requests (in arrival
 * order) as the grids ("slots") of one new batched context while the summed
 * vof_estimate_bytes of the live contexts fits the budget, and advances
 * every live context by one step (one captured CUDA graph per context on
 * its own stream; every slot with its own field, time and step; a slot
 * whose request is done moves no more). A context is freed when all its
 * requests are done. Each result equals the request run alone (vof_init +
 * vof_step with the same CFL), bit for bit.
 * budget_bytes: device memory the contexts may hold (0: 80% of the free
 * memory at creation). max_batch: requests per admitted batch (0: no
 * limit). reserved: zero. */
typedef struct vof_server vof_server;
typedef struct {
  int64_t budget_bytes;
  int32_t precision;
  int32_t flux_polyhedron;
  int32_t reconstruction;
  int32_t max_batch;
  int32_t reserved[2];
} vof_server_options;
typedef struct {
  int64_t n_submitted, n_queued, n_active, n_done;
  int64_t cell_steps;        /* cells x steps of the done requests */
  int64_t device_bytes;      /* held by the live contexts */
  int64_t peak_device_bytes;
  int64_t budget_bytes;
  int64_t n_batches;         /* contexts created */
  int64_t max_active;        /* most requests advanced in one tick */
  double p50_latency_s, p99_latency_s;  /* submit -> result, done requests */
  double elapsed_s;          /* first submit -> last result */
  int64_t batch_steps;       /* steps launched: one graph launch per live batch per tick */
} vof_server_stats;
enum { VOF_REQ_QUEUED = 0, VOF_REQ_RUNNING = 1, VOF_REQ_DONE = 2 };
vof_status vof_server_create(const vof_server_options* opt, vof_server** out);
/* copies the request (HOST mesh arrays and F0 [n_cell]); *id identifies it.
 * The mesh's structure is checked here (VOF_EINVAL); its derived
 * connectivity, and with it the request's exact device footprint, is built
 * once when the request reaches the front of the queue and handed on to
 * its batched context. A mesh the library cannot take (a cell too large)
 * is refused there: vof_server_step returns VOF_EINVAL once, and
 * vof_server_poll of the request returns VOF_EINVAL with the reason. */
vof_status vof_server_submit(vof_server* s, const vof_mesh_desc* mesh, const double* F0,
                             const vof_velocity* vel, int32_t n_steps, double cfl, double t_end,
                             int64_t* id);
/* one scheduling tick; *n_active (may be NULL): requests advanced. VOF_ENOMEM
 * if the first queued request alone exceeds the budget. */
vof_status vof_server_step(vof_server* s, int32_t* n_active);
/* ticks until every submitted request is done */
vof_status vof_server_drain(vof_server* s);
/* *state: VOF_REQ_*; when done, F (HOST [n_cell], may be NULL) receives the
 * result and *latency_s (may be NULL) the submit-to-result time (-1 before) */
vof_status vof_server_poll(vof_server* s, int64_t id, int32_t* state, double* F,
                           double* latency_s);
vof_status vof_server_get_stats(vof_server* s, vof_server_stats* out);
void vof_server_destroy(vof_server* s);

#ifdef __cplusplus
}
#endif
#endif
