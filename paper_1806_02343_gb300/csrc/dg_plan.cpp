// Host-side mesh planning of dynamic regridding (Sec. 5). The new mesh is kept
// as one state per old leaf (kept, refined, or member of a coarsened group), so
// that a point lookup is a search over the old leaves' Morton codes and the new
// leaves come out in Morton order by walking the old ones.
#include "dg_plan.h"

#include <algorithm>
#include <numeric>
#include <thread>
#include <utility>

#include "../../include/dg_mhd.h"

namespace dgmhd {

namespace {

constexpr int kMaxLevel = 17;  // levels a context accepts (coordinates fit 18 bits)

// spread the low 21 bits of x to every third bit (bit b -> bit 3b)
inline uint64_t spread3(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
// spread the low 32 bits of x to every second bit
inline uint64_t spread2(uint64_t x) {
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
// Morton code of the lower corner of the cube (l, k) at resolution R >= l
inline uint64_t morton(int D, int R, int l, const int32_t* k) {
  const int sh = R - l;
  if (D == 3)
    return spread3((uint64_t)k[0] << sh) | (spread3((uint64_t)k[1] << sh) << 1) |
           (spread3((uint64_t)k[2] << sh) << 2);
  return spread2((uint64_t)k[0] << sh) | (spread2((uint64_t)k[1] << sh) << 1);
}

// largest position p with start[p] <= c (start[0] == 0 <= c), searched outwards
// from the hint: neighbour queries land near the asking leaf in Morton order
inline int64_t locate(const std::vector<uint64_t>& st, uint64_t c, int64_t h) {
  const int64_t N = (int64_t)st.size();
  int64_t lo, hi;
  if (st[h] <= c) {
    lo = h;
    for (int64_t step = 1;; step <<= 1) {
      hi = lo + step;
      if (hi >= N) {
        hi = N;
        break;
      }
      if (st[hi] > c) break;
      lo = hi;
    }
  } else {
    hi = h;
    for (int64_t step = 1;; step <<= 1) {
      lo = hi - step;
      if (lo <= 0) {
        lo = 0;
        break;
      }
      if (st[lo] <= c) break;
      hi = lo;
    }
  }
  while (hi - lo > 1) {  // st[lo] <= c < st[hi] (hi == N: past the end)
    const int64_t mid = lo + (hi - lo) / 2;
    if (st[mid] <= c)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

inline uint64_t leaf_key(int l, const int32_t* k, int D) {
  const uint64_t z = D == 3 ? (uint64_t)k[2] : 0;
  return ((uint64_t)l << 58) | ((uint64_t)k[0] << 38) | ((uint64_t)k[1] << 18) | z;
}

}  // namespace

int morton_index(int D, int64_t N, const int8_t* level, const int32_t* ijk, MortonIndex& mi, bool partial) {
  if ((D != 2 && D != 3) || N < 1 || N > ((int64_t)1 << 30) || !level || !ijk) return DG_E_ARG;
  mi = MortonIndex{};
  mi.D = D;
  mi.N = N;
  int lmax = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int l = level[i];
    if (l < 0 || l > kMaxLevel) return DG_E_MESH;
    for (int a = 0; a < D; ++a)
      if (ijk[i * D + a] < 0 || ijk[i * D + a] >= (1 << l)) return DG_E_MESH;
    lmax = std::max(lmax, l);
  }
  mi.lmax = lmax;
  mi.R = lmax + 1;
  std::vector<uint64_t> code((size_t)N);
  bool sorted = true;
  for (int64_t i = 0; i < N; ++i) {
    code[i] = morton(D, mi.R, level[i], &ijk[i * D]);
    if (i > 0 && code[i] <= code[i - 1]) sorted = false;
  }
  if (sorted) {
    mi.start.swap(code);
    mi.lev.assign(level, level + N);
  } else {
    mi.at.resize((size_t)N);
    std::iota(mi.at.begin(), mi.at.end(), 0);
    std::sort(mi.at.begin(), mi.at.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
    mi.pos.resize((size_t)N);
    mi.start.resize((size_t)N);
    mi.lev.resize((size_t)N);
    for (int64_t p = 0; p < N; ++p) {
      mi.pos[mi.at[p]] = p;
      mi.start[p] = code[mi.at[p]];
      mi.lev[p] = level[mi.at[p]];
    }
  }
  // the leaves tile the cube iff, in Morton order, each starts where the one
  // before it ends (a leaf of level l spans 2^(D (R - l)) codes) and the last
  // ends at 2^(D R)
  uint64_t next = 0;
  for (int64_t p = 0; p < N; ++p) {
    if (partial ? mi.start[p] < next : mi.start[p] != next) return DG_E_MESH;  // overlap (or a hole)
    next = mi.start[p] + (1ull << (D * (mi.R - mi.lev[p])));
  }
  if (!partial && next != 1ull << (D * mi.R)) return DG_E_MESH;
  return DG_OK;
}

bool mesh_balanced(const MortonIndex& mi, const int32_t* ijk) {
  const int D = mi.D;
  const int lmin = *std::min_element(mi.lev.begin(), mi.lev.end());
  // A face neighbour cube of the same level lying inside a leaf at least two
  // levels coarser is the only way the rule can fail (seen from the finer
  // side). Across a face inside the grandparent the neighbour cube lies in the
  // grandparent, which is split, so only faces on the grandparent's boundary
  // (the side the leaf's and its parent's octant bits both point to) count.
  for (int64_t p = 0; p < mi.N; ++p) {
    const int l = mi.lev[p];
    if (l - 2 < lmin) continue;
    const int32_t* k = &ijk[(int64_t)mi.leaf(p) * D];
    const int32_t n = 1 << l;
    for (int a = 0; a < D; ++a) {
      const int b0 = k[a] & 1, b1 = (k[a] >> 1) & 1;
      if (b0 != b1) continue;
      const int s = b0 ? 1 : -1;
      int32_t nk[3] = {k[0], k[1], D == 3 ? k[2] : 0};
      nk[a] = (nk[a] + s + n) % n;
      if (mi.lev[locate(mi.start, morton(D, mi.R, l, nk), p)] < l - 1) return false;
    }
  }
  return true;
}

int octree_faces(int D, int64_t N, const int8_t* level, const int32_t* ijk, MortonIndex& mi,
                 std::vector<int32_t>& fL, std::vector<int32_t>& fR, std::vector<int32_t>& fmeta,
                 std::vector<int32_t>& cstart, std::vector<int32_t>& centry, int& maxent, bool partial) {
  if (N < 1 || N > ((int64_t)1 << 30)) return DG_E_MESH;
  if (morton_index(D, N, level, ijk, mi, partial) != DG_OK) return DG_E_MESH;
  // the leaf at Morton position q holds the code (always, on a full mesh)
  auto holds = [&](int64_t q, uint64_t code) {
    return mi.start[q] <= code && code - mi.start[q] < (1ull << (D * (mi.R - mi.lev[q])));
  };
  // the faces a leaf lists: same-level faces on its -a sides, coarse-fine
  // faces on the sides with a coarser neighbour (checking the 2:1 rule)
  auto faces_of_leaf = [&](int64_t cidx, std::vector<int32_t>& fL_, std::vector<int32_t>& fR_,
                           std::vector<int32_t>& fm_) -> int {
    const int l = level[cidx];
    const int32_t n = 1 << l;
    const int32_t* k = &ijk[cidx * D];
    const int64_t p = mi.position((int32_t)cidx);
    // When the cell's 2^D siblings are all leaves (a run of its level in Morton
    // order ending the parent's range), the leaf across a face inside the
    // parent is the sibling of octant o ^ (1 << a): no search.
    int oct = 0;
    for (int a = 0; a < D; ++a) oct |= (k[a] & 1) << a;
    const int64_t first = p - oct;
    bool group = l > 0 && first >= 0 && first + (1 << D) <= N;
    for (int o = 0; o < (1 << D) && group; ++o) group = mi.lev[first + o] == l;
    if (partial && group) {
      // on a partial mesh, a run of same-level leaves need not be the siblings
      const uint64_t span = 1ull << (D * (mi.R - l));
      for (int o = 0; o < (1 << D) && group; ++o)
        group = mi.start[first + o] == mi.start[p] - (uint64_t)oct * span + (uint64_t)o * span;
    }
    for (int a = 0; a < D; ++a) {
      int others[2], no = 0;
      for (int b = 0; b < D; ++b)
        if (b != a) others[no++] = b;
      for (int s = -1; s <= 1; s += 2) {
        int64_t q;
        if (group && ((oct >> a) & 1) == (s < 0 ? 1 : 0)) {
          q = first + (oct ^ (1 << a));
        } else {
          // the leaf holding the corner of the same-level neighbour cube
          int32_t nk[3] = {k[0], k[1], D == 3 ? k[2] : 0};
          nk[a] = (nk[a] + s + n) % n;
          const uint64_t code = morton(D, mi.R, l, nk);
          q = locate(mi.start, code, p);
          if (partial && !holds(q, code)) continue;  // no leaf there: a face of a ghost cell
        }
        const int lq = mi.lev[q];
        if (lq == l) {  // same level: listed once, by the right cell
          if (s < 0) {
            fL_.push_back(mi.leaf(q));
            fR_.push_back((int32_t)cidx);
            fm_.push_back(a);
          }
          continue;
        }
        if (lq == l - 1) {  // coarser neighbour: listed by this (fine) cell
          int sub = 0;
          for (int j = 0; j < no; ++j) sub |= (int)(k[others[j]] & 1) << j;
          if (s < 0) {
            fL_.push_back(mi.leaf(q));
            fR_.push_back((int32_t)cidx);
            fm_.push_back(a | (1 << 2) | (sub << 4));
          } else {
            fL_.push_back((int32_t)cidx);
            fR_.push_back(mi.leaf(q));
            fm_.push_back(a | (2 << 2) | (sub << 4));
          }
          continue;
        }
        if (lq < l - 1) return DG_E_MESH;  // two levels coarser
        if (partial) continue;             // finer neighbours list the faces they have
        // split neighbour: its children along the face must be leaves (2:1)
        int32_t nk[3] = {k[0], k[1], D == 3 ? k[2] : 0};
        nk[a] = (nk[a] + s + n) % n;
        for (int t = 0; t < (1 << (D - 1)); ++t) {
          int32_t ch[3] = {2 * nk[0], 2 * nk[1], 2 * nk[2]};
          ch[a] += s < 0 ? 1 : 0;
          for (int j = 0; j < no; ++j) ch[others[j]] += (t >> j) & 1;
          if (mi.lev[locate(mi.start, morton(D, mi.R, l + 1, ch), q)] != l + 1) return DG_E_MESH;
        }
      }
    }
      return DG_OK;
  };
  // The leaves are split into contiguous chunks searched by parallel host
  // threads; each chunk lists its faces in leaf order and the chunks are
  // concatenated in order, so the lists do not depend on the thread count.
  struct Part {
    std::vector<int32_t> L, R, M;
    int err = DG_OK;
  };
  const int64_t kChunk = 1 << 16;
  const int nth = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)std::max(1u, std::thread::hardware_concurrency()), 16, (N + kChunk - 1) / kChunk}));
  std::vector<Part> parts((size_t)nth);
  auto work = [&](int t) {
    Part& P = parts[(size_t)t];
    const int64_t c0 = N * t / nth, c1 = N * (t + 1) / nth;
    P.L.reserve((size_t)((c1 - c0) * D + (c1 - c0) / 2));
    P.R.reserve(P.L.capacity());
    P.M.reserve(P.L.capacity());
    for (int64_t cidx = c0; cidx < c1 && P.err == DG_OK; ++cidx) P.err = faces_of_leaf(cidx, P.L, P.R, P.M);
  };
  {
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
  }
  size_t total = 0;
  for (const Part& P : parts) {
    if (P.err != DG_OK) return P.err;
    total += P.L.size();
  }
  fL.clear();
  fR.clear();
  fmeta.clear();
  fL.reserve(total);
  fR.reserve(total);
  fmeta.reserve(total);
  for (const Part& P : parts) {
    fL.insert(fL.end(), P.L.begin(), P.L.end());
    fR.insert(fR.end(), P.R.begin(), P.R.end());
    fmeta.insert(fmeta.end(), P.M.begin(), P.M.end());
  }
  // per-cell entries in face order (counting sort)
  const int64_t nf = (int64_t)fL.size();
  cstart.assign((size_t)N + 1, 0);
  for (int64_t f = 0; f < nf; ++f) {
    ++cstart[fL[f] + 1];
    ++cstart[fR[f] + 1];
  }
  maxent = 0;
  for (int64_t c = 0; c < N; ++c) {
    maxent = std::max(maxent, cstart[c + 1]);
    cstart[c + 1] += cstart[c];
  }
  centry.assign((size_t)cstart[N], 0);
  std::vector<int32_t> fill(cstart.begin(), cstart.end() - 1);
  for (int64_t f = 0; f < nf; ++f) {
    centry[fill[fL[f]]++] = (int32_t)(f << 1);
    centry[fill[fR[f]]++] = (int32_t)((f << 1) | 1);
  }
  return DG_OK;
}

void sibling_groups(const MortonIndex& mi, const int32_t* ijk, std::vector<int32_t>& groups) {
  const int D = mi.D, no = 1 << D;
  // In Morton order a complete group is a run of 2^D leaves of one level that
  // starts with octant 0: the parent's code range holds nothing else.
  std::vector<std::pair<uint64_t, int64_t>> found;
  for (int64_t p = 0; p + no <= mi.N; ++p) {
    const int l = mi.lev[p];
    if (l == 0) continue;
    const int32_t* k = &ijk[(int64_t)mi.leaf(p) * D];
    bool first = true;
    for (int a = 0; a < D; ++a) first = first && (k[a] & 1) == 0;
    if (!first) continue;
    bool run = true;
    for (int o = 1; o < no && run; ++o) run = mi.lev[p + o] == l;
    if (!run) continue;
    int32_t pk[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) pk[a] = k[a] >> 1;
    found.emplace_back(leaf_key(l - 1, pk, D), p);
    p += no - 1;
  }
  std::sort(found.begin(), found.end());
  groups.resize(found.size() * no);
  for (size_t g = 0; g < found.size(); ++g)
    for (int o = 0; o < no; ++o) groups[g * no + o] = mi.leaf(found[g].second + o);
}

namespace {

enum : uint8_t { kKeep = 0, kRefined = 1, kCoarsened = 2 };

// The new mesh as a state per old leaf (Morton position) and its lookups.
struct NewMesh {
  const MortonIndex& mi;
  const int32_t* ijk;
  std::vector<uint8_t> st;
  int maxnew = 0;  // bound on the finest new level (coarsening only lowers levels)
  NewMesh(const MortonIndex& m, const int32_t* k) : mi(m), ijk(k), st((size_t)m.N, kKeep) {}

  const int32_t* coords(int64_t p) const { return &ijk[(int64_t)mi.leaf(p) * mi.D]; }

  // level of the new leaf that contains the cube (l, k), -1 if the cube is
  // split into finer new leaves (l <= R); q: the old leaf holding its corner
  int cover(int l, const int32_t* k, int64_t hint, int64_t& q) const {
    q = locate(mi.start, morton(mi.D, mi.R, l, k), hint);
    const int nl = mi.lev[q] + (st[q] == kRefined) - (st[q] == kCoarsened);
    return nl <= l ? nl : -1;
  }

  // no face neighbour of the cube (l, k) holds new leaves of level >= l + 2
  bool face_ok(int l, const int32_t* k, int64_t hint) const {
    if (l + 2 > maxnew) return true;
    const int D = mi.D;
    const int32_t n = 1 << l;
    int64_t q;
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        int32_t nk[3] = {k[0], k[1], D == 3 ? k[2] : 0};
        nk[a] = (nk[a] + s + n) % n;
        if (cover(l, nk, hint, q) >= 0) continue;
        // The neighbour is split: its children along the face must be new
        // leaves. Sufficient: no new leaf in its Morton range is finer than
        // l + 1 (the old leaves of the range follow q; a short scan).
        const uint64_t end = morton(D, mi.R, l, nk) + (1ull << (D * (mi.R - l)));
        int64_t r = q, finest = 0;
        for (; r < mi.N && r < q + 16 && mi.start[r] < end; ++r)
          finest = std::max<int64_t>(finest, mi.lev[r] + (st[r] == kRefined) - (st[r] == kCoarsened));
        if ((r == mi.N || mi.start[r] >= end) && finest <= l + 1) continue;
        int others[2], no = 0;
        for (int b = 0; b < D; ++b)
          if (b != a) others[no++] = b;
        for (int t = 0; t < (1 << (D - 1)); ++t) {
          int32_t ck[3] = {2 * nk[0], 2 * nk[1], 2 * nk[2]};
          ck[a] += s < 0 ? 1 : 0;
          for (int j = 0; j < no; ++j) ck[others[j]] += (t >> j) & 1;
          if (cover(l + 1, ck, q, q) < 0) return false;
        }
      }
    return true;
  }
};

}  // namespace

void plan_mesh(const MortonIndex& mi, const int32_t* ijk, const std::vector<int32_t>& groups, const int8_t* marks,
               std::vector<int32_t>& plan) {
  const int D = mi.D, no = 1 << D;
  const int64_t N = mi.N;
  NewMesh m(mi, ijk);
  for (int64_t p = 0; p < N; ++p) {
    if (marks[mi.leaf(p)] == 1 && mi.lev[p] < kMaxLevel) m.st[p] = kRefined;
    m.maxnew = std::max(m.maxnew, mi.lev[p] + (m.st[p] == kRefined));
  }
  // 2:1 balance by refinement of the coarser side. The old mesh is balanced and
  // refinement adds one level, so only a kept leaf next to a refined one can
  // break the rule: a worklist of the coarser face neighbours of every refined
  // leaf (the same fixed point as re-checking every leaf until none changes).
  std::vector<int64_t> work;
  auto push_coarser_neighbours = [&](int64_t p) {
    const int l = mi.lev[p];
    const int32_t* k = m.coords(p);
    const int32_t n = 1 << l;
    int64_t q;
    for (int a = 0; a < D; ++a)
      for (int s = -1; s <= 1; s += 2) {
        int32_t nk[3] = {k[0], k[1], D == 3 ? k[2] : 0};
        nk[a] = (nk[a] + s + n) % n;
        const int lv = m.cover(l, nk, p, q);
        if (lv >= 0 && lv < l) work.push_back(q);
      }
  };
  for (int64_t p = 0; p < N; ++p)
    if (m.st[p] == kRefined) push_coarser_neighbours(p);
  while (!work.empty()) {
    const int64_t q = work.back();
    work.pop_back();
    if (m.st[q] != kKeep || m.face_ok(mi.lev[q], m.coords(q), q)) continue;
    m.st[q] = kRefined;
    push_coarser_neighbours(q);
  }
  // Coarsening where the parent keeps the balance. Coarsening a group only
  // lowers levels, so it never invalidates another group's check and the
  // result does not depend on the order (the least fixed point); finest
  // parents first reach it in one pass, a second pass confirms it.
  const int64_t ngroups = (int64_t)groups.size() / no;
  std::vector<int64_t> cand;
  for (int64_t g = 0; g < ngroups; ++g) {
    bool all = true;
    for (int o = 0; o < no && all; ++o) all = marks[groups[g * no + o]] == -1;
    if (all) cand.push_back(g);
  }
  std::stable_sort(cand.begin(), cand.end(), [&](int64_t a, int64_t b) {
    return mi.lev[mi.position(groups[a * no])] > mi.lev[mi.position(groups[b * no])];
  });
  std::vector<int32_t> gid((size_t)N, -1);  // group index at the position of its octant 0
  for (bool changed = true; changed;) {
    changed = false;
    size_t kept = 0;
    for (size_t c = 0; c < cand.size(); ++c) {
      const int64_t g = cand[c];
      const int64_t p0 = mi.position(groups[g * no]);
      bool intact = true;
      for (int o = 0; o < no && intact; ++o) intact = m.st[p0 + o] == kKeep;
      if (!intact) continue;  // a member was refined for balance: never coarsened
      for (int o = 0; o < no; ++o) m.st[p0 + o] = kCoarsened;
      int32_t pk[3] = {0, 0, 0};
      const int32_t* k = m.coords(p0);
      for (int a = 0; a < D; ++a) pk[a] = k[a] >> 1;
      if (m.face_ok(mi.lev[p0] - 1, pk, p0)) {
        gid[p0] = (int32_t)g;
        changed = true;
      } else {
        for (int o = 0; o < no; ++o) m.st[p0 + o] = kKeep;
        cand[kept++] = g;
      }
    }
    cand.resize(kept);
  }
  // the new leaves in Morton order: children in octant order, a coarsened
  // group's parent at the place of its octant 0
  plan.clear();
  plan.reserve((size_t)N * 6);
  for (int64_t p = 0; p < N; ++p) {
    const int l = mi.lev[p];
    const int32_t* k = m.coords(p);
    const int32_t i = mi.leaf(p);
    if (m.st[p] == kKeep) {
      plan.insert(plan.end(), {l, k[0], k[1], D == 3 ? k[2] : 0, 0, i});
    } else if (m.st[p] == kRefined) {
      for (int o = 0; o < no; ++o) {
        int32_t c[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) c[a] = 2 * k[a] + ((o >> a) & 1);
        plan.insert(plan.end(), {l + 1, c[0], c[1], c[2], 1 | (o << 4), i});
      }
    } else if (gid[p] >= 0) {
      plan.insert(plan.end(), {l - 1, k[0] >> 1, k[1] >> 1, D == 3 ? k[2] >> 1 : 0, 2, gid[p]});
    }
  }
}

}  // namespace dgmhd

// ------------------------------------------------------------------ C ABI

namespace {

int index_checked(int dim, int64_t n, const int8_t* level, const int32_t* ijk, dgmhd::MortonIndex& mi) {
  const int e = dgmhd::morton_index(dim, n, level, ijk, mi);
  if (e) return e;
  return dgmhd::mesh_balanced(mi, ijk) ? DG_OK : DG_E_MESH;
}

}  // namespace

extern "C" int dg_mhd_sibling_groups(int dim, int64_t n, const int8_t* level, const int32_t* ijk, int64_t cap,
                                     int32_t* groups, int64_t* n_groups) {
  if (!n_groups) return DG_E_ARG;
  dgmhd::MortonIndex mi;
  int e = index_checked(dim, n, level, ijk, mi);
  if (e) return e;
  std::vector<int32_t> g;
  dgmhd::sibling_groups(mi, ijk, g);
  const int64_t ng = (int64_t)g.size() >> dim;
  *n_groups = ng;
  if (!groups) return DG_OK;  // size query
  if (cap < ng) return DG_E_ARG;
  std::copy(g.begin(), g.end(), groups);
  return DG_OK;
}

extern "C" int dg_mhd_regrid_plan_mesh(int dim, int64_t n, const int8_t* level, const int32_t* ijk,
                                       const int8_t* marks, int64_t cap, int8_t* new_level, int32_t* new_ijk,
                                       int32_t* src, int64_t* n_new) {
  if (!marks || !n_new) return DG_E_ARG;
  dgmhd::MortonIndex mi;
  int e = index_checked(dim, n, level, ijk, mi);
  if (e) return e;
  for (int64_t i = 0; i < n; ++i)
    if (marks[i] < -1 || marks[i] > 1) return DG_E_ARG;
  std::vector<int32_t> g, plan;
  dgmhd::sibling_groups(mi, ijk, g);
  dgmhd::plan_mesh(mi, ijk, g, marks, plan);
  const int64_t nn = (int64_t)plan.size() / 6;
  *n_new = nn;
  if (!new_level || !new_ijk || !src) return DG_OK;  // size query
  if (cap < nn) return DG_E_ARG;
  for (int64_t i = 0; i < nn; ++i) {
    const int32_t* q = &plan[i * 6];
    new_level[i] = (int8_t)q[0];
    for (int a = 0; a < dim; ++a) new_ijk[i * dim + a] = q[1 + a];
    src[2 * i] = q[4];
    src[2 * i + 1] = q[5];
  }
  return DG_OK;
}

extern "C" int dg_mhd_octree_faces(int dim, int64_t n, const int8_t* level, const int32_t* ijk, int partial,
                                   int64_t cap, int32_t* face_left, int32_t* face_right, int32_t* face_meta,
                                   int64_t* n_faces) {
  if (!n_faces || !level || !ijk) return DG_E_ARG;
  if (dim != 2 && dim != 3) return DG_E_ARG;
  if (partial != 0 && partial != 1) return DG_E_ARG;
  dgmhd::MortonIndex mi;
  std::vector<int32_t> fL, fR, fmeta, cstart, centry;
  int maxent = 0;
  const int e = dgmhd::octree_faces(dim, n, level, ijk, mi, fL, fR, fmeta, cstart, centry, maxent, partial != 0);
  if (e) return e;
  const int64_t nf = (int64_t)fL.size();
  *n_faces = nf;
  if (!face_left || !face_right || !face_meta) return DG_OK;  // size query
  if (cap < nf) return DG_E_ARG;
  std::copy(fL.begin(), fL.end(), face_left);
  std::copy(fR.begin(), fR.end(), face_right);
  std::copy(fmeta.begin(), fmeta.end(), face_meta);
  return DG_OK;
}
