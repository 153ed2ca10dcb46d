// Host-side mesh planning of dynamic regridding (Sec. 5): a Morton index of
// the leaves of a periodic octree (quadtree in 2D), the sibling groups, and
// the new leaf list from refinement / coarsening marks with 2:1 balance.
// Plain C++ (no device code); used by the context's regridding calls and by
// the context-free entry points dg_mhd_sibling_groups / dg_mhd_regrid_plan_mesh.
#pragma once
#include <stdint.h>

#include <vector>

namespace dgmhd {

// The leaves in Morton (Z-curve) order of their lower corners, with those
// corners' Morton codes at resolution level R = (finest level) + 1, one more
// than the finest leaf so that the corners of refined children have codes too.
// Axis 0 is the fastest bit of every D-bit group, so the 2^D children of a cube
// follow each other in octant order o = sum_a bit_a << a.
struct MortonIndex {
  int D = 0, R = 0, lmax = 0;
  int64_t N = 0;
  std::vector<int32_t> at;      // Morton position -> leaf index (empty: given order is Morton order)
  std::vector<int64_t> pos;     // leaf index -> Morton position (empty: identity)
  std::vector<uint64_t> start;  // Morton code of the lower corner of the leaf at each position
  std::vector<int8_t> lev;      // level of the leaf at each position
  int32_t leaf(int64_t p) const { return at.empty() ? (int32_t)p : at[p]; }
  int64_t position(int32_t i) const { return pos.empty() ? (int64_t)i : pos[i]; }
};

// Levels in [0, 17], coordinates in [0, 2^level), the leaves tiling the unit
// cube without overlap: DG_OK, else DG_E_MESH (DG_E_ARG for a bad dim / count).
// partial: the leaves need not cover the cube (a partition's owned and ghost
// leaves); they still must not overlap.
int morton_index(int D, int64_t N, const int8_t* level, const int32_t* ijk, MortonIndex& mi, bool partial = false);

// No two face neighbours differ by more than one level (periodic box).
bool mesh_balanced(const MortonIndex& mi, const int32_t* ijk);

// Faces of an octree mesh for the operator's surface integrals (Sec. 3.5) with
// coarse-fine faces (Sec. 4.4), and the validation of a context's mesh: the
// leaves tile the cube (morton_index) and are 2:1 balanced, else DG_E_MESH.
// Cells in the given order; per cell, axes in order and the lower side first:
// a same-level face is listed by its right cell (fL = left neighbour, fR =
// cell, meta = axis); a coarse-fine face by its fine cell (meta = axis | side
// << 2 | sub-face << 4, side 1 when the coarse cell is on the left, 2 when on
// the right; sub-face = the fine cell's octant bits across the face). cstart /
// centry: per cell its face entries (2 f + (cell is fR)) in face order.
// partial: a partition's local mesh; a face whose neighbour region holds no
// leaf is left out (only ghost cells, whose results are discarded, have such
// faces), and the 2:1 checks apply to the leaves present.
int octree_faces(int D, int64_t N, const int8_t* level, const int32_t* ijk, MortonIndex& mi,
                 std::vector<int32_t>& fL, std::vector<int32_t>& fR, std::vector<int32_t>& fmeta,
                 std::vector<int32_t>& cstart, std::vector<int32_t>& centry, int& maxent, bool partial = false);

// Groups of 2^D sibling leaves (the children of one cube, all leaves), sorted by
// (parent level, parent coordinates); groups[g * 2^D + o] = leaf index of octant o.
void sibling_groups(const MortonIndex& mi, const int32_t* ijk, std::vector<int32_t>& groups);

// New leaves from marks (+1 refine, -1 coarsen, 0 keep; per leaf): refine the
// leaves marked +1 below level 17; refine every kept leaf that has a face
// neighbour two levels finer, until none has; then replace by its parent every
// sibling group whose members are all marked -1 and still leaves, where the
// parent has no face neighbour two levels finer, until no group can be. Output:
// 6 int32 per new leaf in Morton order: level, i, j, k (0 past dim), source
// (0 copy, 1 | octant << 4 prolongation, 2 restriction) and source index (the
// old leaf, or the group index into `groups`).
void plan_mesh(const MortonIndex& mi, const int32_t* ijk, const std::vector<int32_t>& groups, const int8_t* marks,
               std::vector<int32_t>& plan);

}  // namespace dgmhd
