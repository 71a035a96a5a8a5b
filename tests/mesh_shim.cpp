// Test-only C shim over the library's host octree (csrc/mesh.cpp), compiled with g++ by
// tests/test_host_mesh.py so the refine/coarsen planning and the neighbour tables can be
// checked on a machine without a GPU.
#include <string>
#include <vector>

#include "../paper_2607_19277_gb300/csrc/mesh.h"

using namespace agile;

extern "C" {

void* shim_create(const int* base, int max_level, const int* bc) {
  const double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  return new HostMesh(base, max_level, bc, lo, hi);
}

void shim_destroy(void* h) { delete static_cast<HostMesh*>(h); }

int shim_nblocks(void* h) { return (int)static_cast<HostMesh*>(h)->blocks().size(); }

void shim_blocks(void* h, int* out) {   // [n][4]: level, x, y, z
  const auto& b = static_cast<HostMesh*>(h)->blocks();
  for (size_t i = 0; i < b.size(); ++i) {
    out[4 * i] = b[i].lev;
    out[4 * i + 1] = b[i].x;
    out[4 * i + 2] = b[i].y;
    out[4 * i + 3] = b[i].z;
  }
}

// Apply a regrid with the given flags; returns n_refined * 65536 + n_coarsened.
int shim_regrid(void* h, const int* flags) {
  HostMesh* m = static_cast<HostMesh*>(h);
  std::vector<int> f(flags, flags + m->blocks().size());
  RegridPlan p = m->plan(f);
  m->apply(p);
  return p.n_refined * 65536 + p.n_coarsened;
}

int shim_balanced(void* h) { return static_cast<HostMesh*>(h)->balanced() ? 1 : 0; }

// Face table: kind and neighbour ids per block and face: out[n][6][5] = kind, nbr[4].
int shim_faces(void* h, int* out) {
  HostMesh* m = static_cast<HostMesh*>(h);
  const int n = (int)m->blocks().size();
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < 6; ++f) {
      FaceInfo fi = m->face(i, f);
      int* o = out + (i * 6 + f) * 5;
      o[0] = fi.kind;
      for (int q = 0; q < 4; ++q) o[1 + q] = fi.nbr[q];
    }
  std::vector<BlockDesc> d;
  std::vector<GhostTask> g;
  std::vector<FixupTask> x;
  int ns = 0;
  std::string err;
  m->build_descs(&d, &g, &x, &ns, &err);
  return err.empty() ? ns : -1;
}
}
