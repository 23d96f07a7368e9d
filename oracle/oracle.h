/*
 * Oracle for the unsplit geometric VOF step (LSGIR / LSFIR + FMFPA / EMFPA / NMFPA) -- TEST
 * INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU implementation of what one time step computes, used
 * by the tests, the smoke check and the CPU-baseline timing to check the CUDA
 * library. Nothing in the product path may call it. It shares no code with
 * the CUDA path. Every function names the passage of the paper it follows.
 *
 * Geometric conventions (shared with the library by specification only):
 *  - faces are planar polygons whose nodes run counter-clockwise seen from
 *    outside the owner cell (Sec. 3.1), so their right-hand normal leaves the
 *    owner; boundary faces have neighbour = -1;
 *  - the PLIC plane of an interfacial cell is  n.(x - xc) + C = 0  with xc the
 *    cell centroid and n the unit normal pointing into the fluid (Eq. plic-eq);
 *    the fluid is the part of the cell where  n.(x - xc) + C >= 0;
 *  - face fluxes V_d, V_F are positive when they leave the owner (Sec. 2.2).
 */
#ifndef GVOF_ORACLE_H
#define GVOF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_mesh orc_mesh;

/* velocity fields of the test problems (Sec. 4.2): kind 1 = 3D deformation
 * (period T), 2 = rigid rotation about the z-parallel axis through centre
 * with angular rate omega, 3 = uniform translation u0. */
typedef struct {
  int kind;
  int pad;
  double period;
  double omega;
  double center[3];
  double u0[3];
} orc_velocity;

/* Builds the derived connectivity (neigbcell, cell->face, cell->vertex,
 * vertex->cell) and geometry (compgrid) of a face-based mesh; Sec. 3.1.
 * Arrays are copied. Returns NULL on invalid input. */
orc_mesh* orc_mesh_build(int64_t n_vert, const double* X, int64_t n_face,
                         const int64_t* face_ptr, const int32_t* face_vert,
                         const int32_t* owner, const int32_t* neighbour,
                         int64_t n_cell);
void orc_mesh_free(orc_mesh* m);

/* geometry: any output pointer may be NULL */
void orc_geometry(const orc_mesh* m, double* cell_vol, double* cell_cen,
                  double* face_cen, double* face_nrm, double* face_area,
                  double* cell_bbox, uint8_t* cell_convex);
/* neigbcell CSR (cells sharing >= 1 node, self excluded, ascending).
 * Returns the entry count; ptr [n_cell+1] and idx may be NULL. */
int64_t orc_neighbors(const orc_mesh* m, int64_t* ptr, int32_t* idx);
/* candidate (overlap) cells of a face: owner, neighbour and their node
 * neighbours, ascending, unique. Returns the count (<= cap written). */
int orc_candidates(const orc_mesh* m, int64_t face, int32_t* out, int cap);

/* taggrid (Sec. 3.3): cut-off of F, node F* by inverse-distance weighting,
 * node / face / cell tags in {-1, 0, 1}. F is modified in place. */
void orc_taggrid(const orc_mesh* m, double eps, double* F, double* Fnode,
                 int8_t* tag_v, int8_t* tag_f, int8_t* tag_c);

/* lsgir (Sec. 2.1.1): unit normals of the cells with tag 0 (others 0). */
void orc_lsgir(const orc_mesh* m, double beta, const double* F,
               const int8_t* tag_c, double* nrm);

/* volume enforcement (Sec. 2.1): C per tag-0 cell with
 * vol(cell ∩ {n.(x-xc)+C >= 0}) = F V by bisection. Others 0. */
void orc_plane_constant(const orc_mesh* m, const double* F,
                        const int8_t* tag_c, const double* nrm, double* C);
double orc_cell_cut_volume(const orc_mesh* m, int64_t cell, const double n[3],
                           double C);

/* initial fluid body (Sec. 3.2, initfgrid): kind 1 sphere (centre c,
 * radius r), 2 infinite cylinder (axis through c along unit a, radius r),
 * 3 half-space a.(x - c) < 0 (a unit). */
typedef struct {
  int kind;
  int pad;
  double c[3];
  double a[3];
  double r;
} orc_body;

/* initfgrid (Sec. 3.2): F of every cell by refinement, each cell's
 * tetrahedra divided into ndiv^3 pieces on which the fluid is where the
 * linear interpolant of the body's signed distance is negative. */
void orc_initfgrid(const orc_mesh* m, const orc_body* body, int ndiv, double* F);

/* LSFIR (Sec. 2.1.2). orc_plic_centre: vertex average of the PLIC polygon
 * of cell c (edge crossings of n.(x - xc) + C = 0, each edge once, plus
 * cell vertices on the plane); returns the number of points (0: out = xc).
 * orc_lsfir_normals: one least-squares normal update from the PLIC centres
 * xp [3 nc] of the interfacial cells (weights |x_k - x|^-2.5, neighbours
 * valid within 45 degrees); returns the cells that kept their normal.
 * orc_lsfir_accept: acceptance step of outer iteration io (a candidate
 * replaces a normal it turns by less than 30 degrees / io); returns the
 * largest accepted turn.
 * orc_lsfir: outer iteration from the normals in nrm (in/out), at most
 * n_out repetitions, a change accepted below 30 degrees / I_out, stop when
 * no normal turned by tol or more; C [nc] receives the plane constants;
 * returns the iterations done. */
int orc_plic_centre(const orc_mesh* m, int64_t c, const double n[3], double C,
                    double out[3]);
int64_t orc_lsfir_normals(const orc_mesh* m, const int8_t* tag_c, const double* nrm,
                          const double* xp, double* cand);
double orc_lsfir_accept(const orc_mesh* m, const int8_t* tag_c, int io, const double* cand,
                        double* nrm);
int orc_lsfir(const orc_mesh* m, int n_out, double tol, const double* F,
              const int8_t* tag_c, double* nrm, double* C);

void orc_velocity_eval(const orc_velocity* v, const double x[3], double t,
                       double u[3]);

/* FMFPA flux polyhedron of one face (Sec. 2.2.2). verts receives 2I+1
 * points: x_1..x_I, the back-traced x_{I+1}..x_{2I}, the apex. Returns I,
 * or -1 if I > cap_I. *Vd = (u_c.n) A dt. flags bit0: a side plane or line
 * was degenerate and the streak-line point was used; bit1: the back-traced
 * loop was edge-on and the apex could not be placed (lambda = 0). */
int orc_fmfpa(const orc_mesh* m, int64_t face, const orc_velocity* v,
              double t_half, double dt, double* verts, int cap_I, double* Vd,
              int* flags);

/* EMFPA flux polyhedron of one face (Sec. 2.2.1). verts receives 3I+1
 * points: x_1..x_I, the back-traced x_{I+1}..x_{2I} (Eq. streak-line2 with
 * the vertex velocity at t_half), the side-face centres s_1..s_I (vertex
 * average of x_i, x_{i+1}, x_{I+i}, x_{I+i+1}) and the apex. Returns I, or
 * -1 if I > cap_I. *Vd = (u_c.n) A dt. flags bit1: the back-traced loop was
 * edge-on and the apex could not be placed (lambda = 0). */
int orc_emfpa(const orc_mesh* m, int64_t face, const orc_velocity* v,
              double t_half, double dt, double* verts, int cap_I, double* Vd,
              int* flags);

/* NMFPA flux polyhedron of one face (Sec. 2.2.3): verts receives 2I
 * points, x_1..x_I and x_i - dt u_c (u_c the face-centre velocity at
 * t_half). Returns I, or -1 if I > cap_I. *Vd = (u_c.n) A dt; flags = 0. */
int orc_nmfpa(const orc_mesh* m, int64_t face, const orc_velocity* v,
              double t_half, double dt, double* verts, int cap_I, double* Vd,
              int* flags);

/* faceflux (Sec. 3.5 with Sec. 2.2): V_d and V_F for every face, with the
 * flux polyhedra of `method` (0: FMFPA, 1: EMFPA, 2: NMFPA). stats[0] = geometric
 * faces, [1] = degenerate-line fallbacks, [2] = edge-on faces, [3] =
 * (face, cell) truncations evaluated, [4] = floating-point operations of those
 * truncations (op counter of this algorithm). stats has 5 entries. Threads:
 * OpenMP over faces. */
void orc_faceflux(const orc_mesh* m, const orc_velocity* v, double t,
                  double dt, const double* F, const int8_t* tag_f,
                  const int8_t* tag_c, const double* nrm, const double* C,
                  double* Vd, double* VF, int64_t* stats, int method);

/* vofadv (Eq. fnext + the final clip): F updated in place. */
void orc_vofadv(const orc_mesh* m, const double* Vd, const double* VF,
                double* F);

/* time step, Eq. eq:cfl, evaluated at t, refined once against the field at
 * t + dt, and cut to reach t_end. */
double orc_suggest_dt(const orc_mesh* m, const orc_velocity* v, double t,
                      double cfl, double t_end);

/* volume of (P ∩ {a_k.x + b_k > 0, k < n_planes}) for a closed oriented
 * polyhedral surface P given as face loops (winding-number semantics, so P
 * may be non-convex or self-intersecting). planes[4k..4k+3] = (a, b). */
double orc_poly_clip_volume(int n_vert, const double* verts, int n_face,
                            const int* face_ptr, const int* face_idx,
                            int n_planes, const double* planes);

/* signed volume of a closed polyhedral surface (divergence theorem). */
double orc_poly_volume(int n_vert, const double* verts, int n_face,
                       const int* face_ptr, const int* face_idx);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
