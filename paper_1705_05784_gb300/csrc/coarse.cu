// Primal/dual coarse grids and wirebasket ranks (Sec. 3, Fig. 2; Table 2
// distance-based fracture coarsening; Sec. 4.3 vertical extrusion).
//
// Matrix: boxes of C cells per axis; the node line of a block is at
// start + floor(size/2), except that with more than one block the first and
// last node lines sit on the boundary cells.  A cell's rank counts the axes on
// which it lies on a node line (3D: V=3, E=2, F=1, I=0; 2D: that count + 1).
// Fractures: networks are connected components of the x-y projection graph;
// Table 2 runs on each network (start = lowest-index cell of degree 1, else
// the lowest cell; neighbours in ascending index; FIFO queues; a candidate is
// dropped from Q_vertex when its level is lowered).  3D plates of a network
// share one vertical grid of frac_cz layers per block; crossing plates join a
// network only when their layer ranges are equal.
#include <algorithm>
#include <climits>

#include "batch.cuh"

namespace fams {

namespace {

constexpr int BIG = 0x7f7f7f7f;  // memset(0x7f) value used as +infinity

__host__ __device__ inline int node_of(int blk, int nb, int n, int C) {
  if (nb > 1 && blk == 0) return 0;
  if (nb > 1 && blk == nb - 1) return n - 1;
  int start = blk * C;
  int size = min(C, n - start);
  return start + size / 2;
}

__global__ void k_matrix_coarse(const Inst* inst, int B, const int* off_row, long long nrow,
                                int* rank, int* primal) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  int loc = (int)(r - I.row_off);
  if (loc >= I.nm) return;
  int x = loc % I.nx, y = (loc / I.nx) % I.ny, z = loc / (I.nx * I.ny);
  int bx = x / I.cx, by = y / I.cy, bz = (I.dim == 3) ? z / I.cz : 0;
  int cnt = (x == node_of(bx, I.nbx, I.nx, I.cx)) + (y == node_of(by, I.nby, I.ny, I.cy));
  if (I.dim == 3) cnt += (z == node_of(bz, I.nbz, I.nz, I.cz));
  rank[r] = (I.dim == 3) ? cnt : cnt + 1;
  primal[r] = bx + I.nbx * (by + I.nby * bz);
}

__global__ void k_matrix_nodes(const Inst* inst, int B, const int* off_nc, long long ncoarse,
                               int* node_cell) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncoarse) return;
  const Inst& I = inst[find_segment(off_nc, B + 1, g)];
  int c = (int)(g - I.nc_off);
  if (c >= I.ncm) return;
  int bx = c % I.nbx, by = (c / I.nbx) % I.nby, bz = c / (I.nbx * I.nby);
  int x = node_of(bx, I.nbx, I.nx, I.cx), y = node_of(by, I.nby, I.ny, I.cy);
  int z = (I.dim == 3) ? node_of(bz, I.nbz, I.nz, I.cz) : 0;
  node_cell[g] = I.row_off + x + I.nx * (y + I.ny * z);
}

// strike graph: along-strike neighbours + crossings
__global__ void k_strike_deg(const int* f_sfirst, const int* f_ns, long long nfr, long long ns_tot,
                             int* deg) {
  long long gs = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gs >= ns_tot) return;
  int gf = find_segment(f_sfirst, (int)nfr + 1, gs);
  int s = (int)(gs - f_sfirst[gf]);
  deg[gs] = (s > 0) + (s + 1 < f_ns[gf]);
}

// plates of a 3D network share one uniform vertical coarse grid (Sec. 4.3):
// two crossing plates join the strike graph only when their layer ranges are
// equal (their fracture-fracture connections stay in A either way)
__device__ inline bool same_layers(const Inst& I, const int* f_k0, const int* f_nk, int fa, int fb) {
  return I.dim != 3 || (f_k0[fa] == f_k0[fb] && f_nk[fa] == f_nk[fb] && f_nk[fa] > 0);
}

__global__ void k_strike_inter_deg(const Inst* inst, int B, const int* off_pair, long long npair,
                                   const int* hit, const int* sa, const int* sb,
                                   const int* f_sfirst, const int* f_k0, const int* f_nk, int* deg) {
  long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= npair || !hit[gp]) return;
  int ii = find_segment(off_pair, B + 1, gp);
  const Inst& I = inst[ii];
  int q = (int)(gp - off_pair[ii]), a = 0, b = 0, off = 0;
  for (int i = 0; i < I.nfr; ++i) {
    int cnt = I.nfr - 1 - i;
    if (q < off + cnt) { a = i; b = i + 1 + (q - off); break; }
    off += cnt;
  }
  if (!same_layers(I, f_k0, f_nk, I.fr_off + a, I.fr_off + b)) return;
  atomicAdd(&deg[f_sfirst[I.fr_off + a] + sa[gp]], 1);
  atomicAdd(&deg[f_sfirst[I.fr_off + b] + sb[gp]], 1);
}

__global__ void k_strike_fill(const int* f_sfirst, const int* f_ns, long long nfr,
                              long long ns_tot, const int* ptr, int* cursor, int* adj) {
  long long gs = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gs >= ns_tot) return;
  int gf = find_segment(f_sfirst, (int)nfr + 1, gs);
  int s = (int)(gs - f_sfirst[gf]);
  int p = ptr[gs];
  if (s > 0) adj[p++] = (int)gs - 1;
  if (s + 1 < f_ns[gf]) adj[p++] = (int)gs + 1;
  cursor[gs] = p - ptr[gs];
}

__global__ void k_strike_inter_fill(const Inst* inst, int B, const int* off_pair, long long npair,
                                    const int* hit, const int* sa, const int* sb,
                                    const int* f_sfirst, const int* f_k0, const int* f_nk,
                                    const int* ptr, int* cursor, int* adj) {
  long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= npair || !hit[gp]) return;
  int ii = find_segment(off_pair, B + 1, gp);
  const Inst& I = inst[ii];
  int q = (int)(gp - off_pair[ii]), a = 0, b = 0, off = 0;
  for (int i = 0; i < I.nfr; ++i) {
    int cnt = I.nfr - 1 - i;
    if (q < off + cnt) { a = i; b = i + 1 + (q - off); break; }
    off += cnt;
  }
  if (!same_layers(I, f_k0, f_nk, I.fr_off + a, I.fr_off + b)) return;
  int u = f_sfirst[I.fr_off + a] + sa[gp];
  int v = f_sfirst[I.fr_off + b] + sb[gp];
  adj[ptr[u] + atomicAdd(&cursor[u], 1)] = v;
  adj[ptr[v] + atomicAdd(&cursor[v], 1)] = u;
}

// connected components by union-find on lab (the parent array): a union
// links the larger root under the smaller, so each component ends with its
// smallest index as label
__global__ void k_label_init(long long n, int* lab) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lab[i] = (int)i;
}

__device__ inline int lab_find(volatile int* parent, int x) {
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

__global__ void k_label_union(long long n, const int* ptr, const int* adj, int* lab) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  volatile int* parent = lab;
  for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
    int c = adj[p];
    if (c <= i) continue;
    int a = lab_find(parent, (int)i), b = lab_find(parent, c);
    while (a != b) {
      if (a < b) { int t = a; a = b; b = t; }
      int old = atomicCAS(&lab[a], a, b);
      if (old == a) break;
      a = lab_find(parent, old);
      b = lab_find(parent, b);
    }
  }
}

__global__ void k_label_flatten(long long n, int* lab) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  volatile int* parent = lab;
  int x = (int)i;
  while (parent[x] != x) x = parent[x];
  lab[i] = x;
}

__global__ void k_is_root(long long n, const int* lab, int* flag) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (lab[i] == (int)i);
}

__global__ void k_net_of(long long n, const int* lab, const int* rootscan, int* net, int* netcnt,
                         int* net_root) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int id = rootscan[lab[i]];
  net[i] = id;
  atomicAdd(&netcnt[id], 1);
  if (lab[i] == (int)i) net_root[id] = (int)i;
}

__global__ void k_net_start(long long n, const int* ptr, const int* net, int* start) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (ptr[i + 1] - ptr[i] == 1) atomicMin(&start[net[i]], (int)i);
}

__global__ void k_net_layers(const int* f_sfirst, const int* f_k0, const int* f_nk, long long nfr,
                             long long ns_tot, const int* net, int* k0min, int* k0max, int* nkmin,
                             int* nkmax) {
  long long gs = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gs >= ns_tot) return;
  int gf = find_segment(f_sfirst, (int)nfr + 1, gs);
  int n = net[gs];
  atomicMin(&k0min[n], f_k0[gf]);
  atomicMax(&k0max[n], f_k0[gf]);
  atomicMin(&nkmin[n], f_nk[gf]);
  atomicMax(&nkmax[n], f_nk[gf]);
}

// Table 2 on one network (one thread per network).  Q_vertex removals are
// lazy: a removed entry stays in the array with its flag cleared and is skipped
// when extracted, which keeps the order of the remaining entries.
__global__ void k_bfs(long long nnet, const int* net_cell_off, const int* net_start,
                      const int* net_root, const int* net_inst_dmin, const int* ptr,
                      const int* adj, int* level, int* prim, int* inqv, int* qv, int* q1, int* q2,
                      int* vlist, int* nv_out) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnet) return;
  int base = net_cell_off[n];
  int dmin = net_inst_dmin[n];
  int dmax = dmin <= 0 ? INT_MAX : dmin;
  int start = net_start[n] == BIG ? net_root[n] : net_start[n];
  int vh = base, vt = base;
  qv[vt++] = start;
  inqv[start] = 1;
  int nv = 0;
  while (vh < vt) {
    int v = qv[vh++];
    if (!inqv[v]) continue;
    inqv[v] = 0;
    int np = nv++;
    vlist[base + np] = v;
    prim[v] = np;
    level[v] = 0;
    int* A = q1;
    int* Bq = q2;
    int ah = base, at = base;
    A[at++] = v;
    int dist = 1;
    while (dist <= dmax && ah < at) {
      int bt = base;
      while (ah < at) {
        int c = A[ah++];
        for (int p = ptr[c]; p < ptr[c + 1]; ++p) {
          int m = adj[p];
          if (level[m] > dist) {
            inqv[m] = 0;
            level[m] = dist;
            prim[m] = np;
            Bq[bt++] = m;
          }
        }
      }
      int* t = A; A = Bq; Bq = t;
      ah = base;
      at = bt;
      if (dist == INT_MAX) break;
      ++dist;
    }
    if (dist > dmax) {
      for (int k = ah; k < at; ++k) {
        qv[vt++] = A[k];
        inqv[A[k]] = 1;
      }
    }
  }
  nv_out[n] = nv;
}

__device__ inline int frac_row(const Inst& I, int gc) { return I.row_off + I.nm + (gc - I.fc_off); }

__global__ void k_frac_rank(const Inst* inst, int B, const int* off_fr, const int* f_cfirst,
                            const int* f_sfirst, const int* f_ns, const int* f_k0, long long nfr,
                            long long nfc, const int* s_net, const int* s_prim, const int* s_vert,
                            const int* net_nv, const int* net_k0, const int* net_nk,
                            const int* net_base, int* rank, int* primal) {
  long long gc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= nfc) return;
  int gf = find_segment(f_cfirst, (int)nfr + 1, gc);
  const Inst& I = inst[find_segment(off_fr, B + 1, gf)];
  int loc = (int)(gc - f_cfirst[gf]);
  int ns = f_ns[gf];
  int s = loc % ns, kk = loc / ns;
  int gs = f_sfirst[gf] + s;
  int n = s_net[gs];
  int onv = s_vert[gs];
  int r = frac_row(I, (int)gc);
  if (I.dim == 2) {
    rank[r] = onv ? RANK_V : RANK_E;
    primal[r] = net_base[n] + s_prim[gs];
  } else {
    int cz = max(1, I.fcz);
    int nk = net_nk[n];
    int nvb = (nk + cz - 1) / cz;
    int kn = f_k0[gf] + kk - net_k0[n];
    int vb = kn / cz;
    int onl = (kn == node_of(vb, nvb, nk, cz));
    rank[r] = (onv && onl) ? RANK_V : ((onv || onl) ? RANK_E : RANK_F);
    primal[r] = net_base[n] + s_prim[gs] + net_nv[n] * vb;
  }
}

__global__ void k_frac_nodes(const Inst* inst, int B, const int* off_fr, const int* f_cfirst,
                             const int* f_sfirst, const int* f_ns, const int* f_k0, long long nfr,
                             long long nnet, const int* net_cell_off, const int* net_inst,
                             const int* net_nv, const int* net_k0, const int* net_nk,
                             const int* net_base, const int* vlist, int* node_cell) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nnet) return;
  const Inst& I = inst[net_inst[n]];
  int nv = net_nv[n];
  int cz = max(1, I.fcz);
  int nk = I.dim == 3 ? net_nk[n] : 1;
  int nvb = I.dim == 3 ? (nk + cz - 1) / cz : 1;
  for (int vb = 0; vb < nvb; ++vb) {
    int layer = I.dim == 3 ? net_k0[n] + node_of(vb, nvb, nk, cz) : 0;
    for (int j = 0; j < nv; ++j) {
      int v = vlist[net_cell_off[n] + j];
      int gf = find_segment(f_sfirst, (int)nfr + 1, v);
      int s = v - f_sfirst[gf];
      int loc = s + (I.dim == 3 ? f_ns[gf] * (layer - f_k0[gf]) : 0);
      node_cell[I.nc_off + net_base[n] + j + nv * vb] = frac_row(I, f_cfirst[gf] + loc);
    }
  }
}

// rate-controlled wells: one coarse node each after the fracture nodes
// (Sec. 3: a well's DOF maps to the coarse scale by the identity), rank V,
// its own primal block
__global__ void k_well_coarse(const Inst* inst, int B, const int* off_row, long long nrow,
                              int* rank, int* primal, int* node_cell) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  const int k = (int)(r - I.row_off) - I.nm - I.nf;
  if (k < 0) return;
  const int c = I.nc - I.nw + k;
  rank[r] = RANK_V;
  primal[r] = c;
  node_cell[I.nc_off + c] = (int)r;
}

__global__ void k_primal_global(const Inst* inst, int B, const int* off_row, long long nrow,
                                const int* primal, int* gprimal, int* iota) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > nrow) return;
  iota[r] = (int)r;
  if (r == nrow) return;
  const Inst& I = inst[find_segment(off_row, B + 1, r)];
  gprimal[r] = I.nc_off + primal[r];
}

}  // namespace

int phase_coarse(Batch& b) {
  const int T = 256;
  cudaStream_t st = b.stream;
  long long nrow = b.tot_row, ns = b.tot_s, nfr = b.tot_fr, np = b.tot_pair, nfc = b.tot_fc;
  // matrix blocks
  for (auto& I : b.h) {
    I.nbx = (I.nx + I.cx - 1) / I.cx;
    I.nby = (I.ny + I.cy - 1) / I.cy;
    I.nbz = I.dim == 3 ? (I.nz + I.cz - 1) / I.cz : 1;
    I.ncm = I.nbx * I.nby * I.nbz;
  }
  FAMS_TRY(b.upload_inst());
  FAMS_TRY(b.alloc((void**)&b.rank, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.alloc((void**)&b.primal, sizeof(int) * (nrow + 1)));
  if (nrow > 0)
    fams::note_launch(), k_matrix_coarse<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, b.rank,
                                                     b.primal);
  // strike graph
  int *deg = nullptr, *sptr = nullptr, *cursor = nullptr, *adj = nullptr;
  FAMS_TRY(b.scratch((void**)&deg, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.scratch((void**)&sptr, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.scratch((void**)&cursor, sizeof(int) * (ns + 1)));
  if (ns > 0) fams::note_launch(), k_strike_deg<<<grid_for(ns, T), T, 0, st>>>(b.f_sfirst, b.f_ns, nfr, ns, deg);
  if (np > 0)
    fams::note_launch(), k_strike_inter_deg<<<grid_for(np, T), T, 0, st>>>(b.d_inst, b.B, b.off_pair, np, b.inter_hit,
                                                      b.inter_sa, b.inter_sb, b.f_sfirst, b.f_k0,
                                                      b.f_nk, deg);
  long long nadj = 0;
  FAMS_TRY(exclusive_scan(b, deg, sptr, ns, &nadj));
  FAMS_TRY(b.scratch((void**)&adj, sizeof(int) * (nadj + 1)));
  if (ns > 0)
    fams::note_launch(), k_strike_fill<<<grid_for(ns, T), T, 0, st>>>(b.f_sfirst, b.f_ns, nfr, ns, sptr, cursor, adj);
  if (np > 0)
    fams::note_launch(), k_strike_inter_fill<<<grid_for(np, T), T, 0, st>>>(b.d_inst, b.B, b.off_pair, np, b.inter_hit,
                                                       b.inter_sa, b.inter_sb, b.f_sfirst, b.f_k0,
                                                       b.f_nk, sptr, cursor, adj);
  FAMS_TRY(sort_segments(b, sptr, (int)ns, adj, nullptr, true));
  // networks
  int *lab = nullptr, *flag = nullptr, *rscan = nullptr;
  FAMS_TRY(b.scratch((void**)&lab, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.scratch((void**)&flag, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.scratch((void**)&rscan, sizeof(int) * (ns + 1)));
  long long nnet = 0;
  if (ns > 0) {
    fams::note_launch(), k_label_init<<<grid_for(ns, T), T, 0, st>>>(ns, lab);
    fams::note_launch(), k_label_union<<<grid_for(ns, T), T, 0, st>>>(ns, sptr, adj, lab);
    fams::note_launch(), k_label_flatten<<<grid_for(ns, T), T, 0, st>>>(ns, lab);
    fams::note_launch(), k_is_root<<<grid_for(ns, T), T, 0, st>>>(ns, lab, flag);
    FAMS_TRY(exclusive_scan(b, flag, rscan, ns, &nnet));
  }
  b.tot_net = nnet;
  FAMS_TRY(b.alloc((void**)&b.s_net, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.alloc((void**)&b.s_prim, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.alloc((void**)&b.s_vert, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.alloc((void**)&b.net_nv, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.alloc((void**)&b.net_k0, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.alloc((void**)&b.net_nk, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.alloc((void**)&b.net_base, sizeof(int) * (nnet + 1)));
  int *netcnt = nullptr, *netoff = nullptr, *nroot = nullptr, *nstart = nullptr;
  int *k0max = nullptr, *nkmax = nullptr, *level = nullptr, *inqv = nullptr;
  int *qv = nullptr, *q1 = nullptr, *q2 = nullptr, *vlist = nullptr, *ndmin = nullptr;
  int* ninst = nullptr;
  FAMS_TRY(b.scratch((void**)&netcnt, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&netoff, sizeof(int) * (nnet + 2)));
  FAMS_TRY(b.scratch((void**)&nroot, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&nstart, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&k0max, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&nkmax, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&ndmin, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&ninst, sizeof(int) * (nnet + 1)));
  FAMS_TRY(b.scratch((void**)&level, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.scratch((void**)&inqv, sizeof(int) * (ns + 1)));
  FAMS_TRY(b.scratch((void**)&qv, sizeof(int) * (ns + nnet + 1)));
  FAMS_TRY(b.scratch((void**)&q1, sizeof(int) * (ns + nnet + 1)));
  FAMS_TRY(b.scratch((void**)&q2, sizeof(int) * (ns + nnet + 1)));
  FAMS_TRY(b.scratch((void**)&vlist, sizeof(int) * (ns + nnet + 1)));
  std::vector<int> h_nv(nnet), h_k0min(nnet), h_k0max(nnet), h_nkmin(nnet), h_nkmax(nnet);
  std::vector<int> h_cnt(nnet), h_netinst(nnet);
  if (nnet > 0) {
    FAMS_CUDA(cudaMemsetAsync(netcnt, 0, sizeof(int) * (nnet + 1), st));
    FAMS_CUDA(cudaMemsetAsync(nstart, 0x7f, sizeof(int) * (nnet + 1), st));
    FAMS_CUDA(cudaMemsetAsync(b.net_k0, 0x7f, sizeof(int) * (nnet + 1), st));
    FAMS_CUDA(cudaMemsetAsync(b.net_nk, 0x7f, sizeof(int) * (nnet + 1), st));
    FAMS_CUDA(cudaMemsetAsync(k0max, 0, sizeof(int) * (nnet + 1), st));
    FAMS_CUDA(cudaMemsetAsync(nkmax, 0, sizeof(int) * (nnet + 1), st));
    fams::note_launch(), k_net_of<<<grid_for(ns, T), T, 0, st>>>(ns, lab, rscan, b.s_net, netcnt, nroot);
    fams::note_launch(), k_net_start<<<grid_for(ns, T), T, 0, st>>>(ns, sptr, b.s_net, nstart);
    fams::note_launch(), k_net_layers<<<grid_for(ns, T), T, 0, st>>>(b.f_sfirst, b.f_k0, b.f_nk, nfr, ns, b.s_net,
                                                b.net_k0, k0max, b.net_nk, nkmax);
    FAMS_CUDA(cudaMemcpyAsync(h_k0min.data(), b.net_k0, sizeof(int) * nnet, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(h_k0max.data(), k0max, sizeof(int) * nnet, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(h_nkmin.data(), b.net_nk, sizeof(int) * nnet, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(h_nkmax.data(), nkmax, sizeof(int) * nnet, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(h_cnt.data(), netcnt, sizeof(int) * nnet, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
  }
  // networks per instance (strike cells of an instance are contiguous)
  std::vector<int> h_rscan(ns + 1, 0);
  if (ns > 0) {
    FAMS_CUDA(cudaMemcpyAsync(h_rscan.data(), rscan, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost,
                              st));
    FAMS_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<int> h_off(nnet + 1, 0), h_dmin(nnet, 0);
  for (long long n = 0; n < nnet; ++n) h_off[n + 1] = h_off[n] + h_cnt[n] + 1;
  for (int i = 0; i < b.B; ++i) {
    Inst& I = b.h[i];
    I.net_off = I.ns ? h_rscan[I.s_off] : (i ? b.h[i - 1].net_off + b.h[i - 1].nnet : 0);
    I.nnet = (I.ns ? h_rscan[I.s_off + I.ns] : I.net_off) - I.net_off;
    for (int n = I.net_off; n < I.net_off + I.nnet; ++n) {
      h_dmin[n] = I.dmin;
      h_netinst[n] = i;
      if (I.dim == 3 && (h_k0min[n] != h_k0max[n] || h_nkmin[n] != h_nkmax[n])) {
        set_error("internal: a fracture network joins plates of different layer ranges");
        return FAMS_EINVAL;
      }
    }
  }
  if (nnet > 0) {
    FAMS_CUDA(cudaMemcpyAsync(netoff, h_off.data(), sizeof(int) * (nnet + 1), cudaMemcpyHostToDevice, st));
    FAMS_CUDA(cudaMemcpyAsync(ndmin, h_dmin.data(), sizeof(int) * nnet, cudaMemcpyHostToDevice, st));
    FAMS_CUDA(cudaMemcpyAsync(ninst, h_netinst.data(), sizeof(int) * nnet, cudaMemcpyHostToDevice, st));
    FAMS_CUDA(cudaMemsetAsync(level, 0x7f, sizeof(int) * (ns + 1), st));
    FAMS_CUDA(cudaMemsetAsync(inqv, 0, sizeof(int) * (ns + 1), st));
    FAMS_CUDA(cudaMemsetAsync(b.s_prim, 0xff, sizeof(int) * (ns + 1), st));
    fams::note_launch(), k_bfs<<<grid_for(nnet, 32), 32, 0, st>>>(nnet, netoff, nstart, nroot, ndmin, sptr, adj, level,
                                             b.s_prim, inqv, qv, q1, q2, vlist, b.net_nv);
    FAMS_CUDA(cudaGetLastError());
    FAMS_CUDA(cudaMemcpyAsync(h_nv.data(), b.net_nv, sizeof(int) * nnet, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
  }
  // vertex flags
  {
    std::vector<int> hv(ns + nnet + 1), hflag(ns + 1, 0);
    if (nnet > 0) {
      FAMS_CUDA(cudaMemcpyAsync(hv.data(), vlist, sizeof(int) * (ns + nnet + 1),
                                cudaMemcpyDeviceToHost, st));
      FAMS_CUDA(cudaStreamSynchronize(st));
    }
    for (long long n = 0; n < nnet; ++n)
      for (int j = 0; j < h_nv[n]; ++j) hflag[hv[h_off[n] + j]] = 1;
    FAMS_CUDA(cudaMemcpyAsync(b.s_vert, hflag.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice,
                              st));
  }
  // coarse numbering
  std::vector<int> h_base(nnet + 1, 0);
  long long nc_tot = 0;
  for (int i = 0; i < b.B; ++i) {
    Inst& I = b.h[i];
    int base = I.ncm;
    for (int n = I.net_off; n < I.net_off + I.nnet; ++n) {
      h_base[n] = base;
      int nvb = 1;
      if (I.dim == 3) {
        int cz = std::max(1, I.fcz);
        nvb = (h_nkmin[n] + cz - 1) / cz;
      }
      base += h_nv[n] * nvb;
    }
    I.nc = base + I.nw;
    I.nc_off = (int)nc_tot;
    nc_tot += I.nc;
  }
  b.tot_nc = nc_tot;
  if (nnet > 0)
    FAMS_CUDA(cudaMemcpyAsync(b.net_base, h_base.data(), sizeof(int) * nnet, cudaMemcpyHostToDevice,
                              st));
  FAMS_TRY(b.upload_inst());
  FAMS_TRY(b.alloc((void**)&b.node_cell, sizeof(int) * (nc_tot + 1)));
  if (nc_tot > 0)
    fams::note_launch(), k_matrix_nodes<<<grid_for(nc_tot, T), T, 0, st>>>(b.d_inst, b.B, b.off_nc, nc_tot, b.node_cell);
  if (nfc > 0)
    fams::note_launch(), k_frac_rank<<<grid_for(nfc, T), T, 0, st>>>(b.d_inst, b.B, b.off_fr, b.f_cfirst, b.f_sfirst,
                                                b.f_ns, b.f_k0, nfr, nfc, b.s_net, b.s_prim,
                                                b.s_vert, b.net_nv, b.net_k0, b.net_nk, b.net_base,
                                                b.rank, b.primal);
  if (nnet > 0)
    fams::note_launch(), k_frac_nodes<<<grid_for(nnet, T), T, 0, st>>>(b.d_inst, b.B, b.off_fr, b.f_cfirst, b.f_sfirst,
                                                  b.f_ns, b.f_k0, nfr, nnet, netoff, ninst,
                                                  b.net_nv, b.net_k0, b.net_nk, b.net_base, vlist,
                                                  b.node_cell);
  if (b.tot_w > 0)
    fams::note_launch(), k_well_coarse<<<grid_for(nrow, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow,
                                                                         b.rank, b.primal, b.node_cell);
  FAMS_CUDA(cudaGetLastError());
  // cells of each primal block (rows of R^FV), sorted
  int *gprim = nullptr, *iota = nullptr;
  FAMS_TRY(b.scratch((void**)&gprim, sizeof(int) * (nrow + 1)));
  FAMS_TRY(b.scratch((void**)&iota, sizeof(int) * (nrow + 2)));
  fams::note_launch(), k_primal_global<<<grid_for(nrow + 1, T), T, 0, st>>>(b.d_inst, b.B, b.off_row, nrow, b.primal,
                                                       gprim, iota);
  FAMS_TRY(transpose(b, iota, gprim, nullptr, (int)nrow, (int)nc_tot, nrow, &b.blk_ptr,
                     &b.blk_cell, nullptr, true));
  FAMS_CUDA(cudaGetLastError());
  return b.check_err("coarse grids");
}

}  // namespace fams
