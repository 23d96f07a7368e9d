// Host-side derived connectivity of a face-based mesh (Sec. 3.1).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace gvof {

struct HostConn {
  std::vector<int64_t> cf_ptr, cv_ptr, vc_ptr, nb_ptr;
  std::vector<int32_t> cf, cv, vc, nb;
  int max_cell_faces, max_cell_verts, max_cell_entries;
};

bool build_connectivity(int64_t nv, int64_t nf, int64_t nc, const int64_t* fptr,
                        const int32_t* fvert, const int32_t* own, const int32_t* nbr,
                        HostConn& out, std::string& err);

// the connectivity of grids joined into one index space (grid g's cells,
// faces and vertices shifted by cell_off[g], face_off[g], vert_off[g]): the
// same arrays build_connectivity makes for the joined mesh, without
// rebuilding them
void join_connectivity(const std::vector<const HostConn*>& parts, const std::vector<int64_t>& cell_off,
                       const std::vector<int64_t>& face_off, const std::vector<int64_t>& vert_off,
                       HostConn& out);

}  // namespace gvof
