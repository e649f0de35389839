// Basis functions and the prolongation P (Sec. 3.1, Eqs. 9-22; Appendix A)
// and truncation (Sec. 4.3).
//
// Vertex rows of P are the Kronecker delta (Eq. 16).  Every other row is
// built stage by stage in wirebasket order; in a stage, each dual block B (a
// connected component of the stage's cells under the kept links) solves
//     A'_BB P_B = sum over kept links to known rows c of T_rc P_c,
// where A' is the fine matrix without Dirichlet terms with every dropped link
// removed from the diagonal.  The coupling strategy decides which links are
// kept (Appendix A):
//   Decoupled: same medium and rank(c) >= rank(r)
//   Frac-AMS : matrix rows also keep all fracture links (fracture rows first)
//   Rock-AMS : fracture rows also keep all matrix links (matrix rows first)
//   Coupled  : rank(c) >= rank(r) in either medium (merged dual blocks)
// A'_BB is a symmetric, diagonally dominant M-matrix, solved densely by
// elimination without pivoting: one warp per small dual block, one CTA per
// larger one.
#include <algorithm>

#include "batch.cuh"
#include "dense.cuh"

namespace fams {

namespace {

constexpr int NSTAGE = 5;
constexpr int HASH_CAP = 2048;      // distinct coarse columns one dual block may touch
constexpr int MEMBER_SORT_MAX = 8192;
constexpr int CTA_WARPS = 4;            // warp-per-block launches: blocks per CTA
constexpr long long WARP_NEED = 1024;   // doubles: largest block solved by one warp
constexpr long long MID_NEED = 6144;    // doubles: largest block on a 128-thread CTA

__device__ inline int stage_of(int variant, int med, int rank) {
  if (rank == RANK_V) return -1;
  switch (variant) {
    case 0:  // Decoupled: [mE] [fE] [mF] [fF] [mI]
      if (med == 0) return rank == RANK_E ? 0 : (rank == RANK_F ? 2 : 4);
      return rank == RANK_E ? 1 : 3;
    case 1:  // Frac-AMS: [fE] [fF] [mE] [mF] [mI]
      if (med == 1) return rank == RANK_E ? 0 : 1;
      return rank == RANK_E ? 2 : (rank == RANK_F ? 3 : 4);
    case 2:  // Rock-AMS: [mE] [mF] [mI] [fE] [fF]
      if (med == 0) return rank == RANK_E ? 0 : (rank == RANK_F ? 1 : 2);
      return rank == RANK_E ? 3 : 4;
    default:  // Coupled: [mE,fE] [mF,fF] [mI]
      return rank == RANK_E ? 0 : (rank == RANK_F ? 1 : 2);
  }
}

// cross: 1 if the link joins fracture cells of two different input fractures
// of one coarsening network, 2 if of two networks.  Faces of different
// fractures meet only along edges: a face-face link across a crossing is never
// kept.  Networks are coarsened apart (3D plates of other layer ranges that
// cross), so no link between two networks is kept: each network's basis
// functions are built on that network alone.
__device__ inline bool keep_link(int variant, int mr, int rr, int mc, int rc, int cross) {
  if (mc == 2) return true;    // a well's value is known (P^ww = I): Eq. 18's beta term
  if (mr == 2) return false;   // well rows are coarse nodes
  if (cross == 2 && mr == 1 && mc == 1) return false;
  if (cross && mr == 1 && mc == 1 && rr == RANK_F && rc == RANK_F) return false;
  switch (variant) {
    case 0: return mr == mc && rc >= rr;
    case 1: return (mr == 0) ? (mc == 1 || rc >= rr) : (mc == 1 && rc >= rr);
    case 2: return (mr == 1) ? (mc == 0 || rc >= rr) : (mc == 0 && rc >= rr);
    default: return rc >= rr;
  }
}

// plate[r]: input fracture of row r (-1 for matrix rows); plate[nrow + r]:
// its coarsening network
__device__ inline int crossing(const int* plate, long long nrow, int r, int c) {
  int a = plate[r], b = plate[c];
  if (a < 0 || b < 0 || a == b) return 0;
  return plate[nrow + r] != plate[nrow + c] ? 2 : 1;
}

// a same-stage link across the media of a Coupled instance with a merge cap:
// left out of the first union, merged within the cap afterwards
__device__ inline bool capped_cross(const Inst& I, int mr, int mc) {
  return I.merge_cap > 0 && mr != mc;
}

// input fracture and coarsening network of every unknown (-1 for matrix cells)
__global__ void k_row_plate(const Inst* inst, int B, const int* off_row, long long nrow,
                            const int* f_cfirst, const int* f_sfirst, const int* f_ns,
                            const int* s_net, long long nfr, int* plate) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  long long loc = r - I.row_off;
  if (loc < I.nm || loc >= I.nm + I.nf) {   // matrix and well rows
    plate[r] = -1;
    plate[nrow + r] = -1;
    return;
  }
  int gc = (int)(I.fc_off + (loc - I.nm));
  int gf = find_segment(f_cfirst, (int)nfr + 1, gc);
  plate[r] = gf;
  plate[nrow + r] = s_net[f_sfirst[gf] + (gc - f_cfirst[gf]) % f_ns[gf]];
}

struct RowCtx {
  const Inst* inst;
  int B;
  const int* off_row;
  const int* rank;
};

__device__ inline const Inst& inst_of(const Inst* inst, int B, const int* off_row, int r) {
  return inst[find_segment(off_row, B + 1, r)];
}

// 0 matrix, 1 fracture, 2 well
__device__ inline int medium_of(const Inst& I, int r) {
  const int loc = r - I.row_off;
  return loc < I.nm ? 0 : (loc < I.nm + I.nf ? 1 : 2);
}

// P staging: each known row points into the pool of the stage that built it
struct Pool {
  const int* col[NSTAGE + 1];
  const double* val[NSTAGE + 1];
};

__global__ void k_vertex_rows(const Inst* inst, int B, const int* off_nc, long long nct,
                              const int* node_cell, int* vcol, double* vval, int* pstage,
                              int* poff, int* plen) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nct) return;
  const Inst& I = inst[find_segment(off_nc, B + 1, g)];
  int v = node_cell[g];
  vcol[g] = (int)(g - I.nc_off);
  vval[g] = 1.0;
  pstage[v] = NSTAGE;
  poff[v] = (int)g;
  plen[v] = 1;
}

__global__ void k_stage_mark(const Inst* inst, int B, const int* off_row, long long nrow,
                             const int* rank, int s, int* label, int* instage) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  int in = stage_of(I.basis, medium_of(I, (int)r), rank[r]) == s;
  instage[r] = in;
  label[r] = in ? (int)r : -1;
}

// Dual blocks of a stage = connected components of its kept links, by
// union-find on `label` used as the parent array (label[r] = r or -1 from
// k_stage_mark).  A union links the larger root under the smaller, so every
// parent is <= its child and each component ends with its smallest row as
// root: the same labels as propagating minima, in two launches.
__device__ inline int uf_find(volatile int* parent, int x) {
  int cur = parent[x];
  if (cur == x) return x;
  int prev = x, next;
  while (cur > (next = parent[cur])) {   // path halving on the way up
    parent[prev] = next;
    prev = cur;
    cur = next;
  }
  return cur;
}

__global__ void k_stage_union(const Inst* inst, int B, const int* off_row, long long nrow,
                              const int* rank, const int* plate, const int* rowptr,
                              const int* col, const int* instage, int* label) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow || !instage[r]) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  int mr = medium_of(I, (int)r), rr = rank[r];
  volatile int* parent = label;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
    int c = col[p];
    if (c <= r || !instage[c]) continue;
    if (capped_cross(I, mr, medium_of(I, c))) continue;   // merged afterwards, within the cap
    if (!keep_link(I.basis, mr, rr, medium_of(I, c), rank[c], crossing(plate, nrow, (int)r, c))) continue;
    int a = uf_find(parent, (int)r), b = uf_find(parent, c);
    while (a != b) {
      if (a < b) { int t = a; a = b; b = t; }   // link the larger root a under b
      int old = atomicCAS(&label[a], a, b);
      if (old == a) break;
      a = uf_find(parent, old);                 // a was no longer a root
      b = uf_find(parent, b);
    }
  }
}

__global__ void k_stage_flatten(long long nrow, const int* instage, int* label) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow || !instage[r]) return;
  volatile int* parent = label;
  int x = (int)r;
  while (parent[x] != x) x = parent[x];
  label[r] = x;
}

// Coupled with a merge cap (Sec. 3.1: the merged blocks may be limited):
// the blocks of each medium come from the union above without the
// cross-medium links; those links then merge blocks one at a time, in the
// order of A's rows and columns, while the merged block stays within the cap.
// csize[root] = cells of the block of `root`
__global__ void k_root_size(long long nrow, const int* instage, const int* label, int* csize) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrow && instage[r]) atomicAdd(&csize[label[r]], 1);
}

// rows of the stage with a kept cross-medium link to a higher row of the stage
__global__ void k_cross_flag(const Inst* inst, int B, const int* off_row, long long nrow,
                             const int* rank, const int* plate, const int* rowptr, const int* col,
                             const int* instage, int* flag) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  flag[r] = 0;
  if (!instage[r]) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  int mr = medium_of(I, (int)r), rr = rank[r];
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
    int c = col[p];
    if (c <= r || !instage[c] || !capped_cross(I, mr, medium_of(I, c))) continue;
    if (keep_link(I.basis, mr, rr, medium_of(I, c), rank[c], crossing(plate, nrow, (int)r, c))) {
      flag[r] = 1;
      return;
    }
  }
}

__global__ void k_compact_rows(long long nrow, const int* flag, const int* pos, int* list) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrow && flag[r]) list[pos[r]] = (int)r;
}

__device__ inline int cap_find(int* parent, int x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

// one thread per instance walks its listed rows in order (the merge order is
// part of the method's result, so it is sequential by design)
__global__ void k_merge_cap(const Inst* inst, int B, const int* off_row, long long nrow,
                            const int* rank, const int* plate, const int* rowptr, const int* col,
                            const int* instage, const int* list, int nlist, int* label,
                            int* csize) {
  int ii = blockIdx.x * blockDim.x + threadIdx.x;
  if (ii >= B) return;
  const Inst& I = inst[ii];
  if (I.merge_cap <= 0 || nlist == 0) return;
  // first listed row of this instance
  int lo = 0, hi = nlist;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (list[mid] < I.row_off) lo = mid + 1; else hi = mid;
  }
  for (int t = lo; t < nlist && list[t] < I.row_off + I.n; ++t) {
    int r = list[t];
    int mr = medium_of(I, r), rr = rank[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int c = col[p];
      if (c <= r || !instage[c] || !capped_cross(I, mr, medium_of(I, c))) continue;
      if (!keep_link(I.basis, mr, rr, medium_of(I, c), rank[c], crossing(plate, nrow, r, c))) continue;
      int a = cap_find(label, r), b = cap_find(label, c);
      if (a == b || csize[a] + csize[b] > I.merge_cap) continue;
      int l = min(a, b), h = max(a, b);
      label[h] = l;
      csize[l] += csize[h];
    }
  }
}

__global__ void k_root_flag(long long nrow, const int* label, int* flag) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrow) flag[r] = (label[r] == (int)r);
}

__global__ void k_comp_size(long long nrow, const int* label, const int* rscan, int* comp_of,
                            int* size) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  int l = label[r];
  if (l < 0) { comp_of[r] = -1; return; }
  int c = rscan[l];
  comp_of[r] = c;
  atomicAdd(&size[c], 1);
}

__global__ void k_comp_place(long long nrow, const int* comp_of, const int* off, int* cursor,
                             int* members) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  int c = comp_of[r];
  if (c < 0) return;
  members[off[c] + atomicAdd(&cursor[c], 1)] = (int)r;
}

__device__ void bitonic_sort_int(int* a, int m) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          if ((a[i] > a[l]) == up) { int t = a[i]; a[i] = a[l]; a[l] = t; }
        }
      }
      __syncthreads();
    }
  }
}

// one CTA per dual block (list[blockIdx.x]): sort its members, then find the
// coarse columns its known neighbours carry.  mode 0 counts them, mode 1
// writes them sorted.  Mode 0 needs a power of two >= the largest block of
// ints of dynamic shared memory.
__global__ void k_comp_cols(const Inst* inst, int B, const int* off_row, const int* rank,
                            const int* plate, long long nrow, const int* rowptr, const int* col,
                            const int* instage, const int* label,
                            const int* comp_off, int* members, int* pos, const int* pstage,
                            const int* poff, const int* plen, Pool pool, int s, int mode,
                            const int* list, int* ncols, const int* colptr, int* colbuf, int* bw,
                            int* err) {
  extern __shared__ int sm[];   // member sort buffer (mode 0), sized by the launch
  __shared__ int hs[HASH_CAP];
  __shared__ int nuniq, known_links, ncand, s_bl, s_bu;
  int c = list[blockIdx.x];
  int a = comp_off[c], n = comp_off[c + 1] - a;
  if (n > MEMBER_SORT_MAX) {
    if (threadIdx.x == 0) atomicCAS(err, 0, DERR_CAPACITY);
    return;
  }
  if (mode == 0) {
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) sm[i] = i < n ? members[a + i] : 0x7fffffff;
    __syncthreads();
    bitonic_sort_int(sm, m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      members[a + i] = sm[i];
      pos[sm[i]] = i;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { nuniq = 0; known_links = 0; ncand = 0; s_bl = 0; s_bu = 0; }
  __syncthreads();
  const Inst& I = inst_of(inst, B, off_row, members[a]);
  // candidate columns (with repeats): the hash table gets twice as many slots;
  // mode 0 also measures the block matrix's bandwidths in member order
  bool over = false;
  int bl = 0, bu = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r = members[a + i];
    int mr = medium_of(I, r), rr = rank[r];
    int cand = 0, links = 0;
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int cc = col[p];
      if (cc == r) continue;
      if (instage[cc]) {
        // a link to another block of the stage (cut by a merge cap) is dropped
        if (mode == 0 && label[cc] == label[r] &&
            keep_link(I.basis, mr, rr, medium_of(I, cc), rank[cc], crossing(plate, nrow, r, cc))) {
          bl = max(bl, i - pos[cc]);
          bu = max(bu, pos[cc] - i);
        }
        continue;
      }
      if (!keep_link(I.basis, mr, rr, medium_of(I, cc), rank[cc], crossing(plate, nrow, r, cc))) continue;
      ++links;
      if (pstage[cc] < 0) { over = true; continue; }
      cand += plen[cc];
    }
    if (links) atomicAdd(&known_links, links);
    if (cand) atomicAdd(&ncand, cand);
  }
  if (over) atomicCAS(err, 0, DERR_INVAL);
  if (mode == 0) {
    atomicMax(&s_bl, bl);
    atomicMax(&s_bu, bu);
  }
  __syncthreads();
  if (mode == 0 && threadIdx.x == 0) {
    bw[2 * c] = s_bl;
    bw[2 * c + 1] = s_bu;
  }
  int H = 32;
  while (H < 2 * ncand && H < HASH_CAP) H <<= 1;
  for (int i = threadIdx.x; i < H; i += blockDim.x) hs[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int r = members[a + i];
    int mr = medium_of(I, r), rr = rank[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int cc = col[p];
      if (cc == r || instage[cc]) continue;
      if (!keep_link(I.basis, mr, rr, medium_of(I, cc), rank[cc], crossing(plate, nrow, r, cc))) continue;
      int st = pstage[cc];
      if (st < 0) continue;
      const int* pc = pool.col[st] + poff[cc];
      for (int q = 0; q < plen[cc]; ++q) {
        int key = pc[q];
        unsigned h = ((unsigned)key * 2654435761u) & (H - 1);
        for (int probe = 0; probe < H; ++probe) {
          int prev = atomicCAS(&hs[h], -1, key);
          if (prev == -1) { atomicAdd(&nuniq, 1); break; }
          if (prev == key) break;
          h = (h + 1) & (H - 1);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && known_links == 0) atomicCAS(err, 0, DERR_FLOATING);
  if (nuniq > H / 2) {
    if (threadIdx.x == 0) atomicCAS(err, 0, DERR_CAPACITY);
    return;
  }
  if (mode == 0) {
    if (threadIdx.x == 0) ncols[c] = nuniq;
    return;
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x)
    if (hs[i] == -1) hs[i] = 0x7fffffff;
  __syncthreads();
  bitonic_sort_int(hs, H);
  for (int i = threadIdx.x; i < nuniq; i += blockDim.x) colbuf[colptr[c] + i] = hs[i];
}

// bitonic sort of a[0..m) (m a power of two) by one warp
__device__ void warp_bitonic_sort(int* a, int m) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < m; i += 32) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          if ((a[i] > a[l]) == up) { int t = a[i]; a[i] = a[l]; a[l] = t; }
        }
      }
      __syncwarp();
    }
  }
}

// The column search of k_comp_cols for dual blocks of at most WCOL_N members,
// one warp per block (list[]), CTA_WARPS blocks per CTA: most dual blocks are
// the 7-cell edges and 49-cell faces of a 2D coarse grid, which left most of
// a 128-thread CTA idle.  The same results: members sorted, the same
// bandwidths and the same sorted column set.  A block with more candidate
// columns than a warp's table holds is flagged in mode 0 (ovf_flag, appended
// to ovf_list) for k_comp_cols, and skipped in mode 1.
constexpr int WCOL_N = 64;    // members of a block on one warp
constexpr int WCOL_H = 512;   // hash slots per warp

__global__ void __launch_bounds__(32 * CTA_WARPS) k_comp_cols_warp(
    const Inst* inst, int B, const int* off_row, const int* rank, const int* plate, long long nrow,
    const int* rowptr, const int* col, const int* instage, const int* label, const int* comp_off,
    int* members, int* pos, const int* pstage, const int* poff, const int* plen, Pool pool,
    int mode, const int* list, int nlist, int* ncols, const int* colptr, int* colbuf, int* bw,
    int* ovf_flag, int* ovf_list, int* ovf_n, int* err) {
  __shared__ int tab[CTA_WARPS][WCOL_H];
  const unsigned FULL = 0xffffffffu;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = blockIdx.x * CTA_WARPS + wi;
  if (li >= nlist) return;
  const int c = list[li];
  if (mode == 1 && ovf_flag[c]) return;
  int* hs = tab[wi];
  const int a = comp_off[c], n = comp_off[c + 1] - a;   // 1 <= n <= WCOL_N
  if (mode == 0) {
    int m = 32;
    while (m < n) m <<= 1;
    for (int i = lane; i < m; i += 32) hs[i] = i < n ? members[a + i] : 0x7fffffff;
    __syncwarp();
    warp_bitonic_sort(hs, m);
    for (int i = lane; i < n; i += 32) {
      members[a + i] = hs[i];
      pos[hs[i]] = i;
    }
    __syncwarp();
  }
  const Inst& I = inst_of(inst, B, off_row, members[a]);
  int cand = 0, links = 0, bl = 0, bu = 0;
  bool over = false;
  for (int i = lane; i < n; i += 32) {
    int r = members[a + i];
    int mr = medium_of(I, r), rr = rank[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int cc = col[p];
      if (cc == r) continue;
      if (instage[cc]) {
        if (mode == 0 && label[cc] == label[r] &&
            keep_link(I.basis, mr, rr, medium_of(I, cc), rank[cc], crossing(plate, nrow, r, cc))) {
          bl = max(bl, i - pos[cc]);
          bu = max(bu, pos[cc] - i);
        }
        continue;
      }
      if (!keep_link(I.basis, mr, rr, medium_of(I, cc), rank[cc], crossing(plate, nrow, r, cc))) continue;
      ++links;
      if (pstage[cc] < 0) { over = true; continue; }
      cand += plen[cc];
    }
  }
  links = __reduce_add_sync(FULL, links);
  const int ncand = __reduce_add_sync(FULL, cand);
  if (__any_sync(FULL, over) && lane == 0) atomicCAS(err, 0, DERR_INVAL);
  if (mode == 0) {
    bl = __reduce_max_sync(FULL, bl);
    bu = __reduce_max_sync(FULL, bu);
    if (lane == 0) {
      bw[2 * c] = bl;
      bw[2 * c + 1] = bu;
    }
  }
  int H = 32;
  while (H < 2 * ncand && H < HASH_CAP) H <<= 1;
  if (H > WCOL_H) {   // mode 0 only: mode 1 skips the flagged blocks
    if (lane == 0) {
      ovf_flag[c] = 1;
      ovf_list[atomicAdd(ovf_n, 1)] = c;
    }
    return;
  }
  for (int i = lane; i < H; i += 32) hs[i] = -1;
  __syncwarp();
  int mine = 0;
  for (int i = lane; i < n; i += 32) {
    int r = members[a + i];
    int mr = medium_of(I, r), rr = rank[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int cc = col[p];
      if (cc == r || instage[cc]) continue;
      if (!keep_link(I.basis, mr, rr, medium_of(I, cc), rank[cc], crossing(plate, nrow, r, cc))) continue;
      int st = pstage[cc];
      if (st < 0) continue;
      const int* pc = pool.col[st] + poff[cc];
      for (int q = 0; q < plen[cc]; ++q) {
        int key = pc[q];
        unsigned h = ((unsigned)key * 2654435761u) & (H - 1);
        for (int probe = 0; probe < H; ++probe) {
          int prev = atomicCAS(&hs[h], -1, key);
          if (prev == -1) { ++mine; break; }
          if (prev == key) break;
          h = (h + 1) & (H - 1);
        }
      }
    }
  }
  __syncwarp();
  const int nuniq = __reduce_add_sync(FULL, mine);
  if (lane == 0 && links == 0) atomicCAS(err, 0, DERR_FLOATING);
  if (nuniq > H / 2) {
    if (lane == 0) atomicCAS(err, 0, DERR_CAPACITY);
    return;
  }
  if (mode == 0) {
    if (lane == 0) ncols[c] = nuniq;
    return;
  }
  for (int i = lane; i < H; i += 32)
    if (hs[i] == -1) hs[i] = 0x7fffffff;
  __syncwarp();
  warp_bitonic_sort(hs, H);
  for (int i = lane; i < nuniq; i += 32) colbuf[colptr[c] + i] = hs[i];
}

__device__ inline int find_col(const int* cols, int k, int key) {
  int lo = 0, hi = k - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = cols[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

struct CompArgs {
  const Inst* inst;
  int B;
  const int* off_row;
  const int* rank;
  const int* plate;          // input fracture per row, then coarsening network per row
  long long nrow;
  const int* rowptr;
  const int* col;
  const double* val;
  const double* TD;
  const int* instage;
  const int* label;          // block root per in-stage row
  const int* comp_list;
  long long ncomp;
  const int* comp_off;
  const int* members;
  const int* pos;
  const int* colptr;
  const int* colbuf;
  const int* bw;             // per block: lower and upper bandwidth in member order
  const long long* pool_off;
  int* pstage;
  int* poff;
  int* plen;
  Pool pool;
  int s;
  int* out_col;
  double* out_val;
  int* err;
};

// one dual block on a thread group: assemble [A'_BB | right-hand sides] in
// band storage, W = bl + bu + 1 band entries then k right-hand sides per row
// (then n doubles of pivot reciprocals), eliminate, write the block's rows of P
template <class G>
__device__ void comp_solve(const CompArgs& a, int c, double* M, int* red) {
  (void)red;
  const int gr = G::rank(), gs = G::size();
  const int a0 = a.comp_off[c], n = a.comp_off[c + 1] - a0;
  const int k = a.colptr[c + 1] - a.colptr[c];
  const int bl = a.bw[2 * c], bu = a.bw[2 * c + 1], W = bl + bu + 1;
  const int ld = W + k;
  const int* cols = a.colbuf + a.colptr[c];
  const Inst& I = inst_of(a.inst, a.B, a.off_row, a.members[a0]);
  for (long long t = gr; t < (long long)n * ld; t += gs) M[t] = 0.0;
  G::sync();
  for (int i = gr; i < n; i += gs) {
    int r = a.members[a0 + i];
    int mr = medium_of(I, r), rr = a.rank[r];
    double* Mi = M + (long long)i * ld;
    double d = 0.0;
    for (int p = a.rowptr[r]; p < a.rowptr[r + 1]; ++p) {
      int cc = a.col[p];
      double av = a.val[p];
      if (cc == r) { d += av - a.TD[r]; continue; }
      double T = -av;
      // kept, unless it leads to another block of the stage (cut by a merge cap)
      if (keep_link(I.basis, mr, rr, medium_of(I, cc), a.rank[cc], crossing(a.plate, a.nrow, r, cc)) &&
          (!a.instage[cc] || a.label[cc] == a.label[r])) {
        if (a.instage[cc]) {
          int pc = a.pos[cc];
          if (pc < 0 || pc >= n || i - pc > bl || pc - i > bu) { atomicCAS(a.err, 0, DERR_INVAL); continue; }
          Mi[pc - i + bl] = av;
        } else {
          int st = a.pstage[cc];
          const int* pc = a.pool.col[st] + a.poff[cc];
          const double* pv = a.pool.val[st] + a.poff[cc];
          for (int q = 0; q < a.plen[cc]; ++q) {
            int j = find_col(cols, k, pc[q]);
            if (j < 0) { atomicCAS(a.err, 0, DERR_INVAL); continue; }
            Mi[W + j] += T * pv[q];
          }
        }
      } else {
        d -= T;
      }
    }
    Mi[bl] = d;
  }
  G::sync();
  if (!ge_solve<G>(M, ld, n, k, bl, bu, M + (long long)n * ld)) {
    if (gr == 0) atomicCAS(a.err, 0, DERR_BREAKDOWN);
    return;
  }
  long long base = a.pool_off[c];
  for (int t = gr; t < n * k; t += gs) {
    int i = t / k, q = t - i * k;
    a.out_col[base + t] = cols[q];
    a.out_val[base + t] = M[(long long)i * ld + W + q];
  }
  for (int i = gr; i < n; i += gs) {
    int r = a.members[a0 + i];
    a.pstage[r] = a.s;
    a.poff[r] = (int)(base + (long long)i * k);
    a.plen[r] = k;
  }
}

// dual blocks of the stage: one warp each (WarpGroup: CTA_WARPS blocks per
// CTA, `slice` doubles of shared memory each) or one CTA each (CtaGroup; in
// shared memory, or in `gwork` with `slice` doubles per CTA)
template <class G>
__global__ void k_comp_solve(CompArgs a, long long slice, double* gwork) {
  extern __shared__ double dsm[];
  __shared__ int red[32];
  const int sub = G::per_warp ? (threadIdx.x >> 5) : 0;
  const long long idx = (long long)blockIdx.x * (G::per_warp ? (blockDim.x >> 5) : 1) + sub;
  if (idx >= a.ncomp) return;
  double* M = gwork ? gwork + (long long)blockIdx.x * slice : dsm + (long long)sub * slice;
  comp_solve<G>(a, a.comp_list[idx], M, red);
}

// Adaptive update (Sec. 3.1: basis functions recomputed only where the
// fine-scale properties change beyond a threshold).  dirty[c] of a dual block
// of the stage: it holds a marked cell, or one of its rows keeps a link to a
// row of an earlier stage that was solved again (rec)
__global__ void k_block_dirty(const Inst* inst, int B, const int* off_row, long long nrow,
                              const int* rank, const int* plate, const int* rowptr,
                              const int* col, const int* instage, const int* comp_of,
                              const int* marked, const int* rec, int* dirty) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow || !instage[r]) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  int d = marked[r];
  const int mr = medium_of(I, (int)r), rr = rank[r];
  for (int p = rowptr[r]; p < rowptr[r + 1] && !d; ++p) {
    const int c = col[p];
    if (c == r || instage[c] || !rec[c]) continue;
    if (keep_link(I.basis, mr, rr, medium_of(I, c), rank[c], crossing(plate, nrow, (int)r, c))) d = 1;
  }
  if (d) dirty[comp_of[r]] = 1;
}

// a block kept as it was: its rows' pool entries from the untruncated P of
// the last build (each row's nonzeros at their columns in the block's
// sorted column list, zeros elsewhere); one thread per row of such blocks
__global__ void k_block_keep(long long nrow, const int* instage, const int* comp_of,
                             const int* dirty, const int* pos, const int* colptr,
                             const int* colbuf, const long long* pool_off, const int* comp_off,
                             const int* oldp, const int* oldc, const double* oldv, int s,
                             int* ocol, double* oval, int* pstage, int* poff, int* plen, int* rec,
                             int* err) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow || !instage[r]) return;
  const int c = comp_of[r];
  if (dirty[c]) {
    rec[r] = 1;
    return;
  }
  const int k = colptr[c + 1] - colptr[c];
  const int* cols = colbuf + colptr[c];
  const long long base = pool_off[c] + (long long)pos[r] * k;
  for (int q = 0; q < k; ++q) {
    ocol[base + q] = cols[q];
    oval[base + q] = 0.0;
  }
  for (int e = oldp[r]; e < oldp[r + 1]; ++e) {
    const int j = find_col(cols, k, oldc[e]);
    if (j < 0) { atomicCAS(err, 0, DERR_INVAL); continue; }
    oval[base + j] = oldv[e];
  }
  pstage[r] = s;
  poff[r] = (int)base;
  plen[r] = k;
  (void)comp_off;
}

// truncation (Sec. 4.3) and CSR of P.  full = true: the basis functions
// before truncation (the flux reconstruction's P).
__device__ inline void trunc_row(const double* pv, int len, double alpha, int* cnt, double* sum,
                                 int* only) {
  int c = 0, amax = -1;
  double s = 0.0, vmax = -1.0;
  for (int q = 0; q < len; ++q) {
    double v = pv[q];
    if (v == 0.0) continue;
    if (fabs(v) > vmax) { vmax = fabs(v); amax = q; }
    if (alpha <= 0.0 || fabs(v) >= alpha) { ++c; s += v; }
  }
  *only = -1;
  if (c == 0 && amax >= 0) { c = 1; s = pv[amax]; *only = amax; }
  *cnt = c;
  *sum = s;
}

__global__ void k_p_count(const Inst* inst, int B, const int* off_row, long long nrow,
                          const int* pstage, const int* poff, const int* plen, Pool pool,
                          bool full, int* cnt) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  int st = pstage[r];
  int c = 0, only;
  double s;
  trunc_row(pool.val[st] + poff[r], plen[r], full ? 0.0 : I.alpha, &c, &s, &only);
  cnt[r] = c;
}

__global__ void k_p_fill(const Inst* inst, int B, const int* off_row, long long nrow,
                         const int* pstage, const int* poff, const int* plen, Pool pool,
                         bool full, const int* p_ptr, int* p_col, double* p_val) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  const double alpha = full ? 0.0 : I.alpha;
  int st = pstage[r];
  const int* pc = pool.col[st] + poff[r];
  const double* pv = pool.val[st] + poff[r];
  int c, only;
  double s;
  trunc_row(pv, plen[r], alpha, &c, &s, &only);
  int o = p_ptr[r];
  if (only >= 0) {
    p_col[o] = pc[only];
    p_val[o] = 1.0;
    return;
  }
  bool scale = alpha > 0.0;
  for (int q = 0; q < plen[r]; ++q) {
    double v = pv[q];
    if (v == 0.0) continue;
    if (alpha <= 0.0 || fabs(v) >= alpha) {
      p_col[o] = pc[q];
      p_val[o] = scale ? v / s : v;
      ++o;
    }
  }
}

__global__ void k_p_global_cols(const Inst* inst, int B, const int* off_row, long long nrow,
                                const int* p_ptr, const int* p_col, int* gcol) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst_of(inst, B, off_row, (int)r);
  for (int p = p_ptr[r]; p < p_ptr[r + 1]; ++p) gcol[p] = I.nc_off + p_col[p];
}

}  // namespace

int phase_basis(Batch& b, const int* marked, int* rec, int* n_solved) {
  const int T = 256;
  const bool adaptive = marked != nullptr;
  if (n_solved) *n_solved = 0;
  cudaStream_t st = b.stream;
  long long nrow = b.tot_row, nct = b.tot_nc;
  int *pstage = nullptr, *poff = nullptr, *plen = nullptr;
  FAMS_TRY(b.scratch((void**)&pstage, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&poff, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&plen, sizeof(int) * (nrow + 1)));
  FAMS_CUDA(cudaMemsetAsync(pstage, 0xff, sizeof(int) * (nrow + 1), st));
  FAMS_CUDA(cudaMemsetAsync(plen, 0, sizeof(int) * (nrow + 1), st));
  Pool pool{};
  int* vcol = nullptr;
  double* vval = nullptr;
  FAMS_TRY(b.scratch((void**)&vcol, sizeof(int) * (nct + 1)));
  FAMS_TRY(b.scratch((void**)&vval, sizeof(double) * (nct + 1)));
  pool.col[NSTAGE] = vcol;
  pool.val[NSTAGE] = vval;
  if (nct > 0)
    fams::note_launch(), k_vertex_rows<<<grid_for(nct, T), T, 0, st>>>(b.d_inst, b.B, b.off_nc, nct, b.node_cell, vcol,
                                                  vval, pstage, poff, plen);
  int* plate = nullptr;
  FAMS_TRY(b.scratch((void**)&plate, sizeof(int) * (2 * nrow + 1)));
  fams::note_launch(), k_row_plate<<<grid_for(nrow, T), T, 0, st>>>(
      b.d_inst, b.B, b.off_row, nrow, b.f_cfirst, b.f_sfirst, b.f_ns, b.s_net, b.tot_fr, plate);
  int *label = nullptr, *instage = nullptr, *flag = nullptr, *rscan = nullptr;
  int *comp_of = nullptr, *pos = nullptr;
  FAMS_TRY(b.scratch((void**)&label, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&instage, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&flag, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&rscan, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&comp_of, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&pos, sizeof(int) * (nrow + 1)));
  bool any_cap = false;
  for (auto& I : b.h) any_cap = any_cap || I.merge_cap > 0;
  int *csize = nullptr, *xlist = nullptr;
  if (any_cap) {
    FAMS_TRY(b.scratch((void**)&csize, sizeof(int) * (nrow + 1)));
    FAMS_TRY(b.scratch((void**)&xlist, sizeof(int) * (nrow + 1)));
  }
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  // leave room for the kernels' static shared memory
  max_smem -= 1024;
  FAMS_CUDA(cudaFuncSetAttribute(k_comp_solve<CtaGroup>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  FAMS_CUDA(cudaFuncSetAttribute(k_comp_solve<WarpGroup>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  for (int s = 0; s < NSTAGE; ++s) {
    fams::note_launch(), k_stage_mark<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, b.rank, s, label,
                                                  instage);
    fams::note_launch(), k_stage_union<<<grid_for(nrow, T), T, 0, st>>>(
        b.d_inst, b.B, b.off_row, nrow, b.rank, plate, b.rowptr, b.col, instage, label);
    fams::note_launch(), k_stage_flatten<<<grid_for(nrow, T), T, 0, st>>>(nrow, instage, label);
    if (any_cap && s < 2) {   // Coupled stages with cross-medium links: [mE,fE], [mF,fF]
      FAMS_CUDA(cudaMemsetAsync(csize, 0, sizeof(int) * (nrow + 1), st));
      fams::note_launch(), k_root_size<<<grid_for(nrow, T), T, 0, st>>>(nrow, instage, label, csize);
      fams::note_launch(), k_cross_flag<<<grid_for(nrow, T), T, 0, st>>>(
          b.d_inst, b.B, b.off_row, nrow, b.rank, plate, b.rowptr, b.col, instage, flag);
      long long nl = 0;
      FAMS_TRY(exclusive_scan(b, flag, rscan, nrow, &nl));
      if (nl > 0) {
        fams::note_launch(), k_compact_rows<<<grid_for(nrow, T), T, 0, st>>>(nrow, flag, rscan, xlist);
        fams::note_launch(), k_merge_cap<<<grid_for(b.B, 32), 32, 0, st>>>(
            b.d_inst, b.B, b.off_row, nrow, b.rank, plate, b.rowptr, b.col, instage, xlist,
            (int)nl, label, csize);
        fams::note_launch(), k_stage_flatten<<<grid_for(nrow, T), T, 0, st>>>(nrow, instage, label);
      }
    }
    fams::note_launch(), k_root_flag<<<grid_for(nrow, T), T, 0, st>>>(nrow, label, flag);
    long long ncomp = 0;
    FAMS_TRY(exclusive_scan(b, flag, rscan, nrow, &ncomp));
    if (ncomp == 0) continue;
    int *size = nullptr, *coff = nullptr, *cursor = nullptr, *members = nullptr;
    int *ncols = nullptr, *colptr = nullptr, *colbuf = nullptr;
    FAMS_TRY(b.scratch((void**)&size, sizeof(int) * (ncomp + 1)));
    FAMS_TRY(b.scratch((void**)&coff, sizeof(int) * (ncomp + 1)));
    FAMS_TRY(b.scratch((void**)&cursor, sizeof(int) * (ncomp + 1)));
    FAMS_TRY(b.scratch((void**)&ncols, sizeof(int) * (ncomp + 1)));
    int* bw = nullptr;
    FAMS_TRY(b.scratch((void**)&bw, sizeof(int) * 2 * (ncomp + 1)));
    FAMS_TRY(b.scratch((void**)&colptr, sizeof(int) * (ncomp + 1)));
    FAMS_CUDA(cudaMemsetAsync(size, 0, sizeof(int) * (ncomp + 1), st));
    FAMS_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (ncomp + 1), st));
    fams::note_launch(), k_comp_size<<<grid_for(nrow, T), T, 0, st>>>(nrow, label, rscan, comp_of, size);
    long long nmem = 0;
    FAMS_TRY(exclusive_scan(b, size, coff, ncomp, &nmem));
    FAMS_TRY(b.scratch((void**)&members, sizeof(int) * (nmem + 1)));
    fams::note_launch(), k_comp_place<<<grid_for(nrow, T), T, 0, st>>>(nrow, comp_of, coff, cursor, members);
    // block sizes on the host: sort buffer of the column search, size classes
    std::vector<int> hs(ncomp), hk(ncomp);
    FAMS_CUDA(cudaMemcpyAsync(hs.data(), size, sizeof(int) * ncomp, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
    int sort_cap = 1, maxn = 0;
    for (int v : hs) maxn = std::max(maxn, v);
    while (sort_cap < maxn) sort_cap <<= 1;
    if (maxn > MEMBER_SORT_MAX) {
      set_error("a dual block has " + std::to_string(maxn) + " cells; at most " +
                std::to_string(MEMBER_SORT_MAX) + " are supported");
      return FAMS_ECAPACITY;
    }
    // column search: blocks of at most WCOL_N members one warp each, the
    // others (and small blocks whose candidates overflow a warp's table) one
    // CTA each
    std::vector<int> lsmall, lbig;
    lsmall.reserve(ncomp);
    lbig.reserve(ncomp);
    for (long long c = 0; c < ncomp; ++c) (hs[c] <= WCOL_N ? lsmall : lbig).push_back((int)c);
    const int nsmall = (int)lsmall.size();
    int nbig = (int)lbig.size();
    int *d_small = nullptr, *d_big = nullptr, *ovf_flag = nullptr, *ovf_n = nullptr;
    FAMS_TRY(b.scratch((void**)&d_small, sizeof(int) * (nsmall + 1)));
    FAMS_TRY(b.scratch((void**)&d_big, sizeof(int) * (ncomp + 1)));   // big, then overflowed small
    FAMS_TRY(b.scratch((void**)&ovf_flag, sizeof(int) * (ncomp + 1)));
    FAMS_TRY(b.scratch((void**)&ovf_n, sizeof(int)));
    if (nsmall)
      FAMS_CUDA(cudaMemcpyAsync(d_small, lsmall.data(), sizeof(int) * nsmall, cudaMemcpyHostToDevice, st));
    if (nbig)
      FAMS_CUDA(cudaMemcpyAsync(d_big, lbig.data(), sizeof(int) * nbig, cudaMemcpyHostToDevice, st));
    FAMS_CUDA(cudaMemsetAsync(ovf_flag, 0, sizeof(int) * (ncomp + 1), st));
    FAMS_CUDA(cudaMemsetAsync(ovf_n, 0, sizeof(int), st));
    if (nsmall)
      fams::note_launch(), k_comp_cols_warp<<<(nsmall + CTA_WARPS - 1) / CTA_WARPS, 32 * CTA_WARPS, 0, st>>>(
          b.d_inst, b.B, b.off_row, b.rank, plate, nrow, b.rowptr, b.col, instage, label, coff,
          members, pos, pstage, poff, plen, pool, 0, d_small, nsmall, ncols, nullptr, nullptr, bw,
          ovf_flag, d_big + nbig, ovf_n, b.d_err);
    if (nbig)
      fams::note_launch(), k_comp_cols<<<nbig, 128, sizeof(int) * sort_cap, st>>>(b.d_inst, b.B, b.off_row, b.rank, plate, nrow, b.rowptr, b.col,
                                            instage, label, coff, members, pos, pstage, poff, plen, pool,
                                            s, 0, d_big, ncols, nullptr, nullptr, bw, b.d_err);
    FAMS_CUDA(cudaGetLastError());
    {
      int h_ovf = 0;
      FAMS_CUDA(cudaMemcpyAsync(&h_ovf, ovf_n, sizeof(int), cudaMemcpyDeviceToHost, st));
      FAMS_CUDA(cudaStreamSynchronize(st));
      if (h_ovf > 0) {
        fams::note_launch(), k_comp_cols<<<h_ovf, 128, sizeof(int) * sort_cap, st>>>(b.d_inst, b.B, b.off_row, b.rank, plate, nrow, b.rowptr, b.col,
                                              instage, label, coff, members, pos, pstage, poff, plen, pool,
                                              s, 0, d_big + nbig, ncols, nullptr, nullptr, bw, b.d_err);
        FAMS_CUDA(cudaGetLastError());
        nbig += h_ovf;
      }
    }
    FAMS_TRY(b.check_err("dual-block columns"));
    long long totc = 0;
    FAMS_TRY(exclusive_scan(b, ncols, colptr, ncomp, &totc));
    FAMS_TRY(b.scratch((void**)&colbuf, sizeof(int) * (totc + 1)));
    if (nsmall)
      fams::note_launch(), k_comp_cols_warp<<<(nsmall + CTA_WARPS - 1) / CTA_WARPS, 32 * CTA_WARPS, 0, st>>>(
          b.d_inst, b.B, b.off_row, b.rank, plate, nrow, b.rowptr, b.col, instage, label, coff,
          members, pos, pstage, poff, plen, pool, 1, d_small, nsmall, ncols, colptr, colbuf, nullptr,
          ovf_flag, nullptr, nullptr, b.d_err);
    if (nbig)
      fams::note_launch(), k_comp_cols<<<nbig, 128, 0, st>>>(b.d_inst, b.B, b.off_row, b.rank, plate, nrow, b.rowptr, b.col,
                                              instage, label, coff, members, pos, pstage, poff, plen, pool,
                                              s, 1, d_big, ncols, colptr, colbuf, nullptr, b.d_err);
    // host plan: pool offsets, and the blocks by size class (doubles of
    // [A'_BB | R]): one warp, a 128-thread CTA, a 256-thread CTA in shared
    // memory, or a 512-thread CTA on a bounded global workspace
    std::vector<int> hbw(2 * ncomp);
    FAMS_CUDA(cudaMemcpyAsync(hk.data(), ncols, sizeof(int) * ncomp, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(hbw.data(), bw, sizeof(int) * 2 * ncomp, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
    std::vector<long long> hpo(ncomp + 1, 0);
    std::vector<int> cls[4];
    long long cmax[4] = {0, 0, 0, 0};
    for (long long c = 0; c < ncomp; ++c) {
      hpo[c + 1] = hpo[c] + (long long)hs[c] * hk[c];
      // band and right-hand sides of every row, pivot reciprocals
      long long need = (long long)hs[c] * ((long long)hbw[2 * c] + hbw[2 * c + 1] + 2 + hk[c]);
      int q = need <= WARP_NEED ? 0 : need <= MID_NEED ? 1 : need * 8 + 1024 <= max_smem ? 2 : 3;
      cls[q].push_back((int)c);
      ++b.class_cnt[q];
      cmax[q] = std::max(cmax[q], need);
    }
    // adaptive update: only the dirty blocks are solved; the others keep the
    // untruncated rows of the last build (pf_*)
    std::vector<int> hdirty;
    int* dirty = nullptr;
    if (adaptive) {
      FAMS_TRY(b.scratch((void**)&dirty, sizeof(int) * (ncomp + 1)));
      FAMS_CUDA(cudaMemsetAsync(dirty, 0, sizeof(int) * (ncomp + 1), st));
      fams::note_launch(), k_block_dirty<<<grid_for(nrow, T), T, 0, st>>>(
          b.d_inst, b.B, b.off_row, nrow, b.rank, plate, b.rowptr, b.col, instage, comp_of,
          marked, rec, dirty);
      hdirty.resize(ncomp);
      FAMS_CUDA(cudaMemcpyAsync(hdirty.data(), dirty, sizeof(int) * ncomp, cudaMemcpyDeviceToHost, st));
      FAMS_CUDA(cudaStreamSynchronize(st));
      for (int q = 0; q < 4; ++q) {
        std::vector<int> keep;
        for (int c : cls[q])
          if (hdirty[c]) keep.push_back(c);
        cls[q].swap(keep);
      }
      for (int q = 0; q < 4; ++q)
        if (n_solved) *n_solved += (int)cls[q].size();
    }
    long long* pool_off = nullptr;
    int* ocol = nullptr;
    double* oval = nullptr;
    int* clist = nullptr;
    FAMS_TRY(b.scratch((void**)&pool_off, sizeof(long long) * (ncomp + 1)));
    FAMS_TRY(b.scratch((void**)&ocol, sizeof(int) * (hpo[ncomp] + 1)));
    FAMS_TRY(b.scratch((void**)&oval, sizeof(double) * (hpo[ncomp] + 1)));
    FAMS_TRY(b.scratch((void**)&clist, sizeof(int) * (ncomp + 1)));
    FAMS_CUDA(cudaMemcpyAsync(pool_off, hpo.data(), sizeof(long long) * (ncomp + 1),
                              cudaMemcpyHostToDevice, st));
    if (hpo[ncomp] > 2147483647LL) {
      set_error("basis stage pool exceeds the int32 index range");
      return FAMS_ECAPACITY;
    }
    pool.col[s] = ocol;
    pool.val[s] = oval;
    if (adaptive)
      fams::note_launch(), k_block_keep<<<grid_for(nrow, T), T, 0, st>>>(
          nrow, instage, comp_of, dirty, pos, colptr, colbuf, pool_off, coff, b.pf_ptr, b.pf_col,
          b.pf_val, s, ocol, oval, pstage, poff, plen, rec, b.d_err);
    CompArgs ca{b.d_inst, b.B, b.off_row, b.rank, plate, nrow, b.rowptr, b.col, b.val, b.TD, instage,
                label, nullptr, 0, coff, members, pos, colptr, colbuf, bw, pool_off, pstage, poff, plen,
                pool, s, ocol, oval, b.d_err};
    // the size classes are disjoint sets of blocks: lists and workspace on the
    // main stream, then each class on its own stream so their tails overlap
    int* lsts[4] = {nullptr, nullptr, nullptr, nullptr};
    long long lo = 0;
    for (int q = 0; q < 4; ++q) {
      if (cls[q].empty()) continue;
      lsts[q] = clist + lo;
      FAMS_CUDA(cudaMemcpyAsync(lsts[q], cls[q].data(), sizeof(int) * cls[q].size(),
                                cudaMemcpyHostToDevice, st));
      lo += (long long)cls[q].size();
    }
    // bounded workspace of the global-memory class: at most ~1 GiB per launch
    const long long per3 = std::max(1LL, (1LL << 27) / std::max(cmax[3], 1LL));
    double* work = nullptr;
    if (!cls[3].empty())
      FAMS_TRY(b.scratch((void**)&work, sizeof(double) * cmax[3] *
                                            std::min(per3, (long long)cls[3].size())));
    cudaStream_t cst[4] = {st, st, st, st};
    FAMS_TRY(fork_streams(b, 3, cst + 1));
    for (int q = 0; q < 4; ++q) {
      if (cls[q].empty()) continue;
      int* lst = lsts[q];
      long long cnt = (long long)cls[q].size();
      cudaStream_t qs = cst[q];
      if (q == 0) {
        long long slice = (cmax[0] + 3) & ~3LL;
        ca.comp_list = lst;
        ca.ncomp = cnt;
        fams::note_launch(),
            k_comp_solve<WarpGroup><<<(int)((cnt + CTA_WARPS - 1) / CTA_WARPS), 32 * CTA_WARPS,
                                      sizeof(double) * slice * CTA_WARPS, qs>>>(ca, slice, nullptr);
      } else if (q < 3) {
        ca.comp_list = lst;
        ca.ncomp = cnt;
        fams::note_launch(),
            k_comp_solve<CtaGroup><<<(int)cnt, q == 1 ? 128 : 256, sizeof(double) * cmax[q], qs>>>(
                ca, cmax[q], nullptr);
      } else {
        for (long long o = 0; o < cnt; o += per3) {
          ca.comp_list = lst + o;
          ca.ncomp = std::min(per3, cnt - o);
          fams::note_launch(),
              k_comp_solve<CtaGroup><<<(int)ca.ncomp, 512, 0, qs>>>(ca, cmax[3], work);
        }
      }
      FAMS_CUDA(cudaGetLastError());
    }
    FAMS_TRY(join_streams(b, 3));
    FAMS_TRY(b.check_err("dual-block solves"));
  }
  // every row must have a basis row
  // P CSR with truncation
  int* cnt = nullptr;
  FAMS_TRY(b.scratch((void**)&cnt, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.alloc((void**)&b.p_ptr, sizeof(int) * (nrow + 1)));
  {
    bool missing = false;
    FAMS_TRY(any_negative(b, pstage, nrow, &missing));
    if (missing) {
      set_error("a cell was left without a basis row (it belongs to no stage)");
      return FAMS_EINVAL;
    }
  }
  fams::note_launch(), k_p_count<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, pstage, poff, plen,
                                             pool, false, cnt);
  long long pnnz = 0;
  FAMS_TRY(exclusive_scan(b, cnt, b.p_ptr, nrow, &pnnz));
  b.tot_pnnz = pnnz;
  FAMS_TRY(b.alloc((void**)&b.p_col, sizeof(int) * (pnnz + 1)));
  FAMS_TRY(b.alloc((void**)&b.p_val, sizeof(double) * (pnnz + 1)));
  fams::note_launch(), k_p_fill<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, pstage, poff, plen,
                                            pool, false, b.p_ptr, b.p_col, b.p_val);
  // the flux reconstruction's P: the basis functions before truncation (the
  // same array when no instance truncates)
  bool any_trunc = false;
  for (auto& I : b.h) any_trunc = any_trunc || I.alpha > 0.0;
  if (any_trunc) {
    FAMS_TRY(b.alloc((void**)&b.pf_ptr, sizeof(int) * (nrow + 1)));
    fams::note_launch(), k_p_count<<<grid_for(nrow, T), T, 0, st>>>(
        b.d_inst, b.B, b.off_row, nrow, pstage, poff, plen, pool, true, cnt);
    long long fnnz = 0;
    FAMS_TRY(exclusive_scan(b, cnt, b.pf_ptr, nrow, &fnnz));
    FAMS_TRY(b.alloc((void**)&b.pf_col, sizeof(int) * (fnnz + 1)));
    FAMS_TRY(b.alloc((void**)&b.pf_val, sizeof(double) * (fnnz + 1)));
    fams::note_launch(), k_p_fill<<<grid_for(nrow, T), T, 0, st>>>(
        b.d_inst, b.B, b.off_row, nrow, pstage, poff, plen, pool, true, b.pf_ptr, b.pf_col,
        b.pf_val);
  } else {
    b.pf_ptr = b.p_ptr;
    b.pf_col = b.p_col;
    b.pf_val = b.p_val;
  }
  b.pf_alias = !any_trunc;
  // P^T with global coarse rows (restriction R^FE and the coarse operator)
  int* gcol = nullptr;
  FAMS_TRY(b.scratch((void**)&gcol, sizeof(int) * (pnnz + 1)));
  fams::note_launch(), k_p_global_cols<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, b.p_ptr,
                                                   b.p_col, gcol);
  FAMS_TRY(transpose(b, b.p_ptr, gcol, b.p_val, (int)nrow, (int)nct, pnnz, &b.pt_ptr, &b.pt_col,
                     &b.pt_val, true));
  FAMS_CUDA(cudaGetLastError());
  return b.check_err("prolongation");
}

}  // namespace fams
