// EDFM geometry on the device (Sec. 2, Eqs. 4-7; intersections Sec. 4.1).
//
// Compiled without fused multiply-add: every expression that decides an
// integer (how many cells a fracture has, which matrix column a piece lies
// in, which cell holds an intersection) is a fixed sequence of correctly
// rounded IEEE-754 double operations, so any conforming implementation that
// evaluates the same sequence reaches the same integers.
//
//  * a fracture segment is clipped to the domain (Liang-Barsky) and cut into
//    n = floor(L/h_f + 1/2) equal cells; a 3D plate is extruded over the
//    layers whose centre lies in [z0, z1);
//  * every fracture cell is split at the grid lines it crosses; each piece
//    lies in the matrix column of its midpoint; pieces in one column are
//    summed; the connection's area is length x depth and its <d> the mean
//    distance from the matrix cell to the fracture line (exact, by clipping);
//  * two crossing fractures get one connection per shared layer between the
//    cells that hold the crossing, T_ab = T_a T_b / (T_a + T_b) with
//    T_a = k_f a_f depth / d_a (the intersection pressure eliminated exactly).
#include "batch.cuh"

namespace fams {

namespace {

constexpr int MAX_BRK = 40;

__global__ void k_frac_clip(const Inst* inst, int B, const int* off_fr, long long nfr,
                            const double* fr, double* seg, int* f_ns, int* f_k0, int* f_nk) {
  long long gf = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gf >= nfr) return;
  const Inst& I = inst[find_segment(off_fr, B + 1, gf)];
  const double* f = fr + 6 * gf;
  double x0 = f[0], y0 = f[1], x1 = f[2], y1 = f[3];
  double lx = (double)I.nx * I.dx, ly = (double)I.ny * I.dy;
  double ddx = x1 - x0, ddy = y1 - y0;
  double t0 = 0.0, t1 = 1.0;
  bool ok = true;
  double ps[4] = {-ddx, ddx, -ddy, ddy};
  double qs[4] = {x0, lx - x0, y0, ly - y0};
  for (int k = 0; k < 4 && ok; ++k) {
    double p = ps[k], q = qs[k];
    if (p == 0.0) {
      if (q < 0.0) ok = false;
      continue;
    }
    double r = q / p;
    if (p < 0.0) {
      if (r > t1) { ok = false; break; }
      if (r > t0) t0 = r;
    } else {
      if (r < t0) { ok = false; break; }
      if (r < t1) t1 = r;
    }
  }
  int ns = 0, k0 = 0, nk = 1;
  double ax = 0, ay = 0, bx = 0, by = 0;
  if (ok) {
    ax = x0 + t0 * ddx; ay = y0 + t0 * ddy;
    bx = x0 + t1 * ddx; by = y0 + t1 * ddy;
    double ex = bx - ax, ey = by - ay;
    double L = sqrt(ex * ex + ey * ey);
    if (L >= ZERO_PIECE * I.hf) {
      ns = (int)floor(L / I.hf + 0.5);
      if (ns < 1) ns = 1;
    }
  }
  if (I.dim == 3) {
    double z0 = f[4], z1 = f[5];
    int first = -1, cnt = 0;
    for (int k = 0; k < I.nz; ++k) {
      double zc = ((double)k + 0.5) * I.dz;
      if (z0 <= zc && zc < z1) {
        if (first < 0) first = k;
        ++cnt;
      }
    }
    if (cnt == 0) ns = 0;
    k0 = first < 0 ? 0 : first;
    nk = ns ? cnt : 0;
  } else {
    nk = ns ? 1 : 0;
  }
  seg[4 * gf + 0] = ax; seg[4 * gf + 1] = ay;
  seg[4 * gf + 2] = bx; seg[4 * gf + 3] = by;
  f_ns[gf] = ns; f_k0[gf] = k0; f_nk[gf] = nk;
}

__device__ inline int floor_div(double v, double h) { return (int)floor(v / h); }

// matrix columns crossed by strike cell s of its fracture, sorted by column
__global__ void k_strike_overlap(const Inst* inst, int B, const int* off_fr, const int* f_sfirst,
                                 long long nfr, long long ns_tot, const double* seg,
                                 const int* f_ns, int* ovcnt, int* ovcol, double* ovlen,
                                 int* err) {
  long long gs = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gs >= ns_tot) return;
  int gf = find_segment(f_sfirst, (int)nfr + 1, gs);
  const Inst& I = inst[find_segment(off_fr, B + 1, gf)];
  int n = f_ns[gf];
  int s = (int)(gs - f_sfirst[gf]);
  double ax = seg[4 * gf], ay = seg[4 * gf + 1], bx = seg[4 * gf + 2], by = seg[4 * gf + 3];
  double ex = bx - ax, ey = by - ay;
  double L = sqrt(ex * ex + ey * ey);
  double ts = (double)s / (double)n, te = (double)(s + 1) / (double)n;
  double brk[MAX_BRK];
  int nb = 0;
  brk[nb++] = ts;
  brk[nb++] = te;
  bool over = false;
  if (ex != 0.0) {
    double xa = ax + ts * ex, xb = ax + te * ex;
    double lo = fmin(xa, xb), hi = fmax(xa, xb);
    for (int i = floor_div(lo, I.dx); i <= floor_div(hi, I.dx) + 1; ++i) {
      double t = ((double)i * I.dx - ax) / ex;
      if (ts < t && t < te) {
        if (nb < MAX_BRK) brk[nb++] = t; else over = true;
      }
    }
  }
  if (ey != 0.0) {
    double ya = ay + ts * ey, yb = ay + te * ey;
    double lo = fmin(ya, yb), hi = fmax(ya, yb);
    for (int j = floor_div(lo, I.dy); j <= floor_div(hi, I.dy) + 1; ++j) {
      double t = ((double)j * I.dy - ay) / ey;
      if (ts < t && t < te) {
        if (nb < MAX_BRK) brk[nb++] = t; else over = true;
      }
    }
  }
  // sort + unique
  for (int i = 1; i < nb; ++i) {
    double v = brk[i];
    int j = i - 1;
    while (j >= 0 && brk[j] > v) { brk[j + 1] = brk[j]; --j; }
    brk[j + 1] = v;
  }
  int m = 0;
  for (int i = 0; i < nb; ++i)
    if (m == 0 || brk[i] != brk[m - 1]) brk[m++] = brk[i];
  int cnt = 0;
  int cols[MAX_OVERLAP];
  double lens[MAX_OVERLAP];
  for (int k = 0; k + 1 < m; ++k) {
    double a = brk[k], c = brk[k + 1];
    double ln = (c - a) * L;
    if (ln < ZERO_PIECE * I.hf) continue;
    double tm = 0.5 * (a + c);
    double px = ax + tm * ex, py = ay + tm * ey;
    int ix = min(max(floor_div(px, I.dx), 0), I.nx - 1);
    int iy = min(max(floor_div(py, I.dy), 0), I.ny - 1);
    int key = ix + I.nx * iy;
    int found = -1;
    for (int q = 0; q < cnt; ++q)
      if (cols[q] == key) found = q;
    if (found >= 0) {
      lens[found] += ln;
    } else if (cnt < MAX_OVERLAP) {
      cols[cnt] = key;
      lens[cnt] = ln;
      ++cnt;
    } else {
      over = true;
    }
  }
  // sort by column
  for (int i = 1; i < cnt; ++i) {
    int c = cols[i];
    double l = lens[i];
    int j = i - 1;
    while (j >= 0 && cols[j] > c) { cols[j + 1] = cols[j]; lens[j + 1] = lens[j]; --j; }
    cols[j + 1] = c;
    lens[j + 1] = l;
  }
  if (over) atomicCAS(err, 0, DERR_CAPACITY);
  ovcnt[gs] = cnt;
  for (int q = 0; q < cnt; ++q) {
    ovcol[gs * MAX_OVERLAP + q] = cols[q];
    ovlen[gs * MAX_OVERLAP + q] = lens[q];
  }
}

// <d>: mean distance from the matrix cell to the fracture line (Eq. 7).  The
// signed distance f = n . (x - A) is linear: over a triangle its integral is
// the area times the mean of f at the corners.  With P+ the part of the cell
// where f >= 0 (the rectangle clipped by that half-plane),
// int |f| = 2 int_{P+} f - area f(centre).  Coordinates relative to the
// cell's lower-left corner; one thread per (strike piece, matrix cell).
__device__ inline double mean_dist_cell(double nx, double ny, double ox, double oy, double dx,
                                        double dy) {
  const double rx[4] = {0.0, dx, dx, 0.0}, ry[4] = {0.0, 0.0, dy, dy};
  double px[5], py[5];
  int m = 0;
  for (int k = 0; k < 4; ++k) {
    int k1 = (k + 1) & 3;
    double fp = nx * (rx[k] - ox) + ny * (ry[k] - oy);
    double fq = nx * (rx[k1] - ox) + ny * (ry[k1] - oy);
    if (fp >= 0.0) { px[m] = rx[k]; py[m] = ry[k]; ++m; }
    if ((fp >= 0.0) != (fq >= 0.0)) {
      double t = fp / (fp - fq);
      px[m] = rx[k] + t * (rx[k1] - rx[k]);
      py[m] = ry[k] + t * (ry[k1] - ry[k]);
      ++m;
    }
  }
  double pos = 0.0;
  for (int k = 1; k + 1 < m; ++k) {
    double area = 0.5 * ((px[k] - px[0]) * (py[k + 1] - py[0]) - (px[k + 1] - px[0]) * (py[k] - py[0]));
    double f1 = nx * (px[0] - ox) + ny * (py[0] - oy);
    double f2 = nx * (px[k] - ox) + ny * (py[k] - oy);
    double f3 = nx * (px[k + 1] - ox) + ny * (py[k + 1] - oy);
    pos += area * (f1 + f2 + f3) / 3.0;
  }
  double A = dx * dy;
  double fc = nx * (0.5 * dx - ox) + ny * (0.5 * dy - oy);
  return (2.0 * pos - A * fc) / A;
}

__global__ void k_mean_dist(const Inst* inst, int B, const int* off_fr, const int* f_sfirst,
                            long long nfr, long long ns_tot, const double* seg,
                            const int* ovcnt, const int* ovcol, double* ovdist) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long gs = id / MAX_OVERLAP;
  int q = (int)(id % MAX_OVERLAP);
  if (gs >= ns_tot || q >= ovcnt[gs]) return;
  int gf = find_segment(f_sfirst, (int)nfr + 1, gs);
  const Inst& I = inst[find_segment(off_fr, B + 1, gf)];
  double ax = seg[4 * gf], ay = seg[4 * gf + 1], bx = seg[4 * gf + 2], by = seg[4 * gf + 3];
  double ex = bx - ax, ey = by - ay;
  double L = sqrt(ex * ex + ey * ey);
  double nx = -ey / L, ny = ex / L;
  int key = ovcol[gs * MAX_OVERLAP + q];
  int ix = key % I.nx, iy = key / I.nx;
  double x0 = (double)ix * I.dx, y0 = (double)iy * I.dy;
  ovdist[gs * MAX_OVERLAP + q] = mean_dist_cell(nx, ny, ax - x0, ay - y0, I.dx, I.dy);
}

// per fracture cell: number of matrix-fracture connections
__global__ void k_cell_nnc_count(const Inst* inst, int B, const int* off_fc, const int* off_fr,
                                 const int* f_cfirst, const int* f_sfirst, const int* f_ns,
                                 long long nfr, long long nfc, const int* ovcnt, int* cnt) {
  long long gc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= nfc) return;
  int gf = find_segment(f_cfirst, (int)nfr + 1, gc);
  int loc = (int)(gc - f_cfirst[gf]);
  int s = loc % f_ns[gf];
  cnt[gc] = ovcnt[f_sfirst[gf] + s];
}

__global__ void k_cell_nnc_fill(const Inst* inst, int B, const int* off_fr, const int* f_cfirst,
                                const int* f_sfirst, const int* f_ns, const int* f_k0,
                                long long nfr, long long nfc, const int* ovcnt, const int* ovcol,
                                const double* ovlen, const double* ovdist, const double* perm,
                                const int* nnc_first, int* nrow_f, int* nrow_m, double* nT,
                                double* narea, double* ndist) {
  long long gc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= nfc) return;
  int gf = find_segment(f_cfirst, (int)nfr + 1, gc);
  const Inst& I = inst[find_segment(off_fr, B + 1, gf)];
  int loc = (int)(gc - f_cfirst[gf]);
  int ns = f_ns[gf];
  int s = loc % ns, kk = loc / ns;
  long long gs = f_sfirst[gf] + s;
  int k = (I.dim == 3) ? f_k0[gf] + kk : 0;
  int frow = I.row_off + I.nm + (int)(gc - I.fc_off);
  int base = nnc_first[gc];
  for (int q = 0; q < ovcnt[gs]; ++q) {
    int m = ovcol[gs * MAX_OVERLAP + q] + I.nx * I.ny * k;
    double area = ovlen[gs * MAX_OVERLAP + q] * I.dz;
    double d = ovdist[gs * MAX_OVERLAP + q];
    nrow_f[base + q] = frow;
    nrow_m[base + q] = I.row_off + m;
    narea[base + q] = area;
    ndist[base + q] = d;
    nT[base + q] = area / d * perm[I.m_off + m];
  }
}

__device__ inline void pair_of(int q, int nfr, int* a, int* b) {
  int off = 0;
  for (int i = 0; i < nfr; ++i) {
    int cnt = nfr - 1 - i;
    if (q < off + cnt) { *a = i; *b = i + 1 + (q - off); return; }
    off += cnt;
  }
  *a = 0; *b = 0;
}

// one thread per fracture pair of an instance: crossing test (closed segments)
__global__ void k_intersect(const Inst* inst, int B, const int* off_pair, long long npair,
                            const double* seg, const int* f_ns, const int* f_k0, const int* f_nk,
                            const double* kf, int* hit, int* sa_out, int* sb_out, double* T_out,
                            int* nlink) {
  long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= npair) return;
  int ii = find_segment(off_pair, B + 1, gp);
  const Inst& I = inst[ii];
  int a, b;
  pair_of((int)(gp - off_pair[ii]), I.nfr, &a, &b);
  int fa = I.fr_off + a, fb = I.fr_off + b;
  hit[gp] = 0;
  nlink[gp] = 0;
  int na = f_ns[fa], nb = f_ns[fb];
  if (na == 0 || nb == 0) return;
  const double* A = seg + 4 * fa;
  const double* C = seg + 4 * fb;
  double d1x = A[2] - A[0], d1y = A[3] - A[1];
  double d2x = C[2] - C[0], d2y = C[3] - C[1];
  double den = d1x * d2y - d1y * d2x;
  double n1 = sqrt(d1x * d1x + d1y * d1y);
  double n2 = sqrt(d2x * d2x + d2y * d2y);
  if (fabs(den) <= 1e-14 * n1 * n2) return;
  double wx = C[0] - A[0], wy = C[1] - A[1];
  double t = (wx * d2y - wy * d2x) / den;
  double u = (wx * d1y - wy * d1x) / den;
  if (!(0.0 <= t && t <= 1.0 && 0.0 <= u && u <= 1.0)) return;
  int sa = min((int)floor(t * na), na - 1);
  int sb = min((int)floor(u * nb), nb - 1);
  double da = fmax(fabs(t - ((double)sa + 0.5) / na) * n1, DIST_FLOOR * I.hf);
  double db = fmax(fabs(u - ((double)sb + 0.5) / nb) * n2, DIST_FLOOR * I.hf);
  double Ta = kf[fa] * I.aperture * I.dz / da;
  double Tb = kf[fb] * I.aperture * I.dz / db;
  int links = 1;
  if (I.dim == 3) {
    int lo = max(f_k0[fa], f_k0[fb]);
    int hi = min(f_k0[fa] + f_nk[fa], f_k0[fb] + f_nk[fb]);
    links = max(0, hi - lo);
    if (links == 0) return;
  }
  hit[gp] = 1;
  sa_out[gp] = sa;
  sb_out[gp] = sb;
  T_out[gp] = Ta * Tb / (Ta + Tb);
  nlink[gp] = links;
}

// fracture-fracture links keyed by their lower cell: along strike, vertical
// (3D), and intersections (placed afterwards)
__global__ void k_ff_count(const Inst* inst, int B, const int* off_fr, const int* f_cfirst,
                           const int* f_ns, const int* f_nk, long long nfr, long long nfc,
                           int* cnt) {
  long long gc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= nfc) return;
  int gf = find_segment(f_cfirst, (int)nfr + 1, gc);
  int loc = (int)(gc - f_cfirst[gf]);
  int ns = f_ns[gf], nk = f_nk[gf];
  int s = loc % ns, kk = loc / ns;
  int c = 0;
  if (s + 1 < ns) ++c;
  if (kk + 1 < nk) ++c;
  cnt[gc] = c;
}

__global__ void k_ff_inter_count(const Inst* inst, int B, const int* off_pair, long long npair,
                                 const int* hit, const int* sa, const int* f_cfirst,
                                 const int* f_ns, const int* f_k0, const int* f_nk, int* cnt) {
  long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= npair || !hit[gp]) return;
  int ii = find_segment(off_pair, B + 1, gp);
  const Inst& I = inst[ii];
  int a, b;
  pair_of((int)(gp - off_pair[ii]), I.nfr, &a, &b);
  int fa = I.fr_off + a, fb = I.fr_off + b;
  int lo = 0, hi = 1;
  if (I.dim == 3) {
    lo = max(f_k0[fa], f_k0[fb]);
    hi = min(f_k0[fa] + f_nk[fa], f_k0[fb] + f_nk[fb]);
  }
  for (int k = lo; k < hi; ++k) {
    int ca = f_cfirst[fa] + sa[gp] + f_ns[fa] * (I.dim == 3 ? k - f_k0[fa] : 0);
    atomicAdd(&cnt[ca], 1);
  }
}

__global__ void k_ff_fill_fixed(const Inst* inst, int B, const int* off_fr, const int* f_cfirst,
                                const int* f_ns, const int* f_nk, const double* seg,
                                const double* kf, long long nfr, long long nfc,
                                const int* ff_first, int* cursor, int* ffa, int* ffb,
                                double* ffT) {
  long long gc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= nfc) return;
  int gf = find_segment(f_cfirst, (int)nfr + 1, gc);
  const Inst& I = inst[find_segment(off_fr, B + 1, gf)];
  int loc = (int)(gc - f_cfirst[gf]);
  int ns = f_ns[gf], nk = f_nk[gf];
  int s = loc % ns, kk = loc / ns;
  double ex = seg[4 * gf + 2] - seg[4 * gf], ey = seg[4 * gf + 3] - seg[4 * gf + 1];
  double h = sqrt(ex * ex + ey * ey) / (double)ns;
  int row = I.row_off + I.nm + (int)(gc - I.fc_off);
  int p = ff_first[gc];
  if (s + 1 < ns) {
    ffa[p] = row; ffb[p] = row + 1; ffT[p] = kf[gf] * I.aperture * I.dz / h; ++p;
  }
  if (kk + 1 < nk) {
    ffa[p] = row; ffb[p] = row + ns; ffT[p] = kf[gf] * I.aperture * h / I.dz; ++p;
  }
  cursor[gc] = p - ff_first[gc];
}

__global__ void k_ff_fill_inter(const Inst* inst, int B, const int* off_pair, long long npair,
                                const int* hit, const int* sa, const int* sb, const double* T,
                                const int* f_cfirst, const int* f_ns, const int* f_k0,
                                const int* f_nk, const int* ff_first, int* cursor, int* ffa,
                                int* ffb, double* ffT) {
  long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= npair || !hit[gp]) return;
  int ii = find_segment(off_pair, B + 1, gp);
  const Inst& I = inst[ii];
  int a, b;
  pair_of((int)(gp - off_pair[ii]), I.nfr, &a, &b);
  int fa = I.fr_off + a, fb = I.fr_off + b;
  int lo = 0, hi = 1;
  if (I.dim == 3) {
    lo = max(f_k0[fa], f_k0[fb]);
    hi = min(f_k0[fa] + f_nk[fa], f_k0[fb] + f_nk[fb]);
  }
  for (int k = lo; k < hi; ++k) {
    int ca = f_cfirst[fa] + sa[gp] + f_ns[fa] * (I.dim == 3 ? k - f_k0[fa] : 0);
    int cb = f_cfirst[fb] + sb[gp] + f_ns[fb] * (I.dim == 3 ? k - f_k0[fb] : 0);
    int p = ff_first[ca] + atomicAdd(&cursor[ca], 1);
    ffa[p] = I.row_off + I.nm + (ca - I.fc_off);
    ffb[p] = I.row_off + I.nm + (cb - I.fc_off);
    ffT[p] = T[gp];
  }
}

// links of one cell sorted by their higher cell (few entries per cell)
__global__ void k_ff_sort_cell(const int* ff_first, long long nfc, int* ffb, double* ffT) {
  long long gc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= nfc) return;
  int a = ff_first[gc], e = ff_first[gc + 1];
  for (int i = a + 1; i < e; ++i) {
    int kb = ffb[i];
    double t = ffT[i];
    int j = i - 1;
    while (j >= a && ffb[j] > kb) { ffb[j + 1] = ffb[j]; ffT[j + 1] = ffT[j]; --j; }
    ffb[j + 1] = kb;
    ffT[j + 1] = t;
  }
}

}  // namespace

int phase_geometry(Batch& b) {
  const int T = 256;
  cudaStream_t st = b.stream;
  long long nfr = b.tot_fr;
  FAMS_TRY(b.alloc((void**)&b.seg, sizeof(double) * 4 * (nfr + 1)));
  FAMS_TRY(b.alloc((void**)&b.f_ns, sizeof(int) * (nfr + 1)));
  FAMS_TRY(b.alloc((void**)&b.f_k0, sizeof(int) * (nfr + 1)));
  FAMS_TRY(b.alloc((void**)&b.f_nk, sizeof(int) * (nfr + 1)));
  FAMS_TRY(b.alloc((void**)&b.f_cfirst, sizeof(int) * (nfr + 1)));
  FAMS_TRY(b.alloc((void**)&b.f_sfirst, sizeof(int) * (nfr + 1)));
  if (nfr > 0)
    fams::note_launch(), k_frac_clip<<<grid_for(nfr, T), T, 0, st>>>(b.d_inst, b.B, b.off_fr, nfr, b.fracs, b.seg,
                                                b.f_ns, b.f_k0, b.f_nk);
  FAMS_CUDA(cudaGetLastError());
  // per-fracture counts to the host: fracture-cell and strike offsets
  std::vector<int> ns(nfr), nk(nfr), k0(nfr);
  if (nfr > 0) {
    FAMS_CUDA(cudaMemcpyAsync(ns.data(), b.f_ns, sizeof(int) * nfr, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(nk.data(), b.f_nk, sizeof(int) * nfr, cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaMemcpyAsync(k0.data(), b.f_k0, sizeof(int) * nfr, cudaMemcpyDeviceToHost, st));
  }
  FAMS_CUDA(cudaStreamSynchronize(st));
  std::vector<int> cfirst(nfr + 1), sfirst(nfr + 1);
  long long c = 0, s = 0;
  for (int i = 0; i < b.B; ++i) {
    Inst& I = b.h[i];
    I.fc_off = (int)c;
    I.s_off = (int)s;
    for (int f = I.fr_off; f < I.fr_off + I.nfr; ++f) {
      cfirst[f] = (int)c;
      sfirst[f] = (int)s;
      c += (long long)ns[f] * (I.dim == 3 ? nk[f] : (ns[f] ? 1 : 0));
      s += ns[f];
    }
    I.nf = (int)(c - I.fc_off);
    I.ns = (int)(s - I.s_off);
  }
  cfirst[nfr] = (int)c;
  sfirst[nfr] = (int)s;
  b.tot_fc = c;
  b.tot_s = s;
  FAMS_CUDA(cudaMemcpyAsync(b.f_cfirst, cfirst.data(), sizeof(int) * (nfr + 1),
                            cudaMemcpyHostToDevice, st));
  FAMS_CUDA(cudaMemcpyAsync(b.f_sfirst, sfirst.data(), sizeof(int) * (nfr + 1),
                            cudaMemcpyHostToDevice, st));
  // rows: matrix cells, fracture cells, then rate-controlled wells per instance
  long long row = 0, pairs = 0;
  for (int i = 0; i < b.B; ++i) {
    Inst& I = b.h[i];
    I.n = I.nm + I.nf + I.nw;
    I.row_off = (int)row;
    row += I.n;
    I.inter_off = (int)pairs;
    I.ninter = I.nfr * (I.nfr - 1) / 2;
    pairs += I.ninter;
  }
  b.tot_row = row;
  b.tot_pair = pairs;
  FAMS_TRY(b.upload_inst());

  // overlaps of strike cells with matrix columns
  long long nsl = b.tot_s;
  FAMS_TRY(b.scratch((void**)&b.s_ovcnt, sizeof(int) * (nsl + 1)));
  FAMS_TRY(b.scratch((void**)&b.s_ovcol, sizeof(int) * MAX_OVERLAP * (nsl + 1)));
  FAMS_TRY(b.scratch((void**)&b.s_ovlen, sizeof(double) * MAX_OVERLAP * (nsl + 1)));
  FAMS_TRY(b.scratch((void**)&b.s_ovdist, sizeof(double) * MAX_OVERLAP * (nsl + 1)));
  if (nsl > 0) {
    fams::note_launch(), k_strike_overlap<<<grid_for(nsl, 128), 128, 0, st>>>(b.d_inst, b.B, b.off_fr, b.f_sfirst, nfr,
                                                         nsl, b.seg, b.f_ns, b.s_ovcnt, b.s_ovcol,
                                                         b.s_ovlen, b.d_err);
    fams::note_launch(), k_mean_dist<<<grid_for(nsl * MAX_OVERLAP, 128), 128, 0, st>>>(
        b.d_inst, b.B, b.off_fr, b.f_sfirst, nfr, nsl, b.seg, b.s_ovcnt, b.s_ovcol, b.s_ovdist);
  }
  FAMS_CUDA(cudaGetLastError());
  FAMS_TRY(b.check_err("fracture clipping"));

  // matrix-fracture connections, ordered by (fracture cell, matrix cell)
  long long nfc = b.tot_fc;
  int* cnt = nullptr;
  FAMS_TRY(b.scratch((void**)&cnt, sizeof(int) * (nfc + 1)));
  FAMS_TRY(b.alloc((void**)&b.nnc_first, sizeof(int) * (nfc + 1)));
  int* nnc_first = b.nnc_first;
  if (nfc > 0)
    fams::note_launch(), k_cell_nnc_count<<<grid_for(nfc, T), T, 0, st>>>(b.d_inst, b.B, b.off_fc, b.off_fr,
                                                     b.f_cfirst, b.f_sfirst, b.f_ns, nfr, nfc,
                                                     b.s_ovcnt, cnt);
  long long nnc = 0;
  FAMS_TRY(exclusive_scan(b, cnt, nnc_first, nfc, &nnc));
  b.tot_nnc = nnc;
  FAMS_TRY(b.alloc((void**)&b.nnc_row_f, sizeof(int) * (nnc + 1)));
  FAMS_TRY(b.alloc((void**)&b.nnc_row_m, sizeof(int) * (nnc + 1)));
  FAMS_TRY(b.alloc((void**)&b.nnc_T, sizeof(double) * (nnc + 1)));
  FAMS_TRY(b.alloc((void**)&b.nnc_area, sizeof(double) * (nnc + 1)));
  FAMS_TRY(b.alloc((void**)&b.nnc_dist, sizeof(double) * (nnc + 1)));
  if (nfc > 0)
    fams::note_launch(), k_cell_nnc_fill<<<grid_for(nfc, T), T, 0, st>>>(
        b.d_inst, b.B, b.off_fr, b.f_cfirst, b.f_sfirst, b.f_ns, b.f_k0, nfr, nfc, b.s_ovcnt,
        b.s_ovcol, b.s_ovlen, b.s_ovdist, b.perm, nnc_first, b.nnc_row_f, b.nnc_row_m, b.nnc_T,
        b.nnc_area, b.nnc_dist);
  FAMS_CUDA(cudaGetLastError());
  // per-instance NNC offsets
  {
    std::vector<int> hf(nfc + 1);
    FAMS_CUDA(cudaMemcpyAsync(hf.data(), nnc_first, sizeof(int) * (nfc + 1),
                              cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < b.B; ++i) {
      Inst& I = b.h[i];
      I.nnc_off = hf[I.fc_off];
      I.nnc = hf[I.fc_off + I.nf] - I.nnc_off;
    }
  }

  // intersections
  long long np = b.tot_pair;
  FAMS_TRY(b.scratch((void**)&b.inter_hit, sizeof(int) * (np + 1)));
  FAMS_TRY(b.scratch((void**)&b.inter_sa, sizeof(int) * (np + 1)));
  FAMS_TRY(b.scratch((void**)&b.inter_sb, sizeof(int) * (np + 1)));
  FAMS_TRY(b.scratch((void**)&b.inter_T, sizeof(double) * (np + 1)));
  int* nlink = nullptr;
  FAMS_TRY(b.scratch((void**)&nlink, sizeof(int) * (np + 1)));
  if (np > 0)
    fams::note_launch(), k_intersect<<<grid_for(np, T), T, 0, st>>>(b.d_inst, b.B, b.off_pair, np, b.seg, b.f_ns,
                                               b.f_k0, b.f_nk, b.kf, b.inter_hit, b.inter_sa,
                                               b.inter_sb, b.inter_T, nlink);
  // fracture-fracture links keyed by the lower cell
  int* ffcnt = nullptr;
  int* cursor = nullptr;
  FAMS_TRY(b.scratch((void**)&ffcnt, sizeof(int) * (nfc + 1)));
  FAMS_TRY(b.alloc((void**)&b.ff_first, sizeof(int) * (nfc + 1)));
  int* ff_first = b.ff_first;
  FAMS_TRY(b.scratch((void**)&cursor, sizeof(int) * (nfc + 1)));
  if (nfc > 0)
    fams::note_launch(), k_ff_count<<<grid_for(nfc, T), T, 0, st>>>(b.d_inst, b.B, b.off_fr, b.f_cfirst, b.f_ns,
                                               b.f_nk, nfr, nfc, ffcnt);
  if (np > 0)
    fams::note_launch(), k_ff_inter_count<<<grid_for(np, T), T, 0, st>>>(b.d_inst, b.B, b.off_pair, np, b.inter_hit,
                                                    b.inter_sa, b.f_cfirst, b.f_ns, b.f_k0,
                                                    b.f_nk, ffcnt);
  long long nff = 0;
  FAMS_TRY(exclusive_scan(b, ffcnt, ff_first, nfc, &nff));
  b.tot_ff = nff;
  FAMS_TRY(b.alloc((void**)&b.ff_a, sizeof(int) * (nff + 1)));
  FAMS_TRY(b.alloc((void**)&b.ff_b, sizeof(int) * (nff + 1)));
  FAMS_TRY(b.alloc((void**)&b.ff_T, sizeof(double) * (nff + 1)));
  if (nfc > 0) {
    fams::note_launch(), k_ff_fill_fixed<<<grid_for(nfc, T), T, 0, st>>>(b.d_inst, b.B, b.off_fr, b.f_cfirst, b.f_ns,
                                                    b.f_nk, b.seg, b.kf, nfr, nfc, ff_first,
                                                    cursor, b.ff_a, b.ff_b, b.ff_T);
    if (np > 0)
      fams::note_launch(), k_ff_fill_inter<<<grid_for(np, T), T, 0, st>>>(b.d_inst, b.B, b.off_pair, np, b.inter_hit,
                                                     b.inter_sa, b.inter_sb, b.inter_T,
                                                     b.f_cfirst, b.f_ns, b.f_k0, b.f_nk,
                                                     ff_first, cursor, b.ff_a, b.ff_b, b.ff_T);
    fams::note_launch(), k_ff_sort_cell<<<grid_for(nfc, T), T, 0, st>>>(ff_first, nfc, b.ff_b, b.ff_T);
  }
  FAMS_CUDA(cudaGetLastError());
  {
    std::vector<int> hf(nfc + 1);
    FAMS_CUDA(cudaMemcpyAsync(hf.data(), ff_first, sizeof(int) * (nfc + 1),
                              cudaMemcpyDeviceToHost, st));
    FAMS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < b.B; ++i) {
      Inst& I = b.h[i];
      I.ff_off = hf[I.fc_off];
      I.nff = hf[I.fc_off + I.nf] - I.ff_off;
    }
  }
  FAMS_TRY(b.upload_inst());
  return b.check_err("fracture geometry");
}

}  // namespace fams
