// Device-wide helpers used by the setup phases: exclusive scan and a CSR
// transpose whose segments come out sorted (deterministic, no atomics in the
// final order).
#include <algorithm>

#include "batch.cuh"

namespace fams {

namespace {

constexpr int SCAN_BLOCK = 1024;

__device__ inline int warp_incl_scan(int v) {
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += t;
  }
  return v;
}

// inclusive scan of one block's values (blockDim.x == SCAN_BLOCK)
__device__ inline int block_incl_scan(int v, int* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_incl_scan(v);
  if (lane == 31) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (SCAN_BLOCK >> 5)) ? sh[lane] : 0;
    s = warp_incl_scan(s);
    sh[lane] = s;
  }
  __syncthreads();
  if (w > 0) v += sh[w - 1];
  __syncthreads();
  return v;
}

__global__ void k_scan_blocks(const int* in, long long n, long long* block_sums) {
  __shared__ int sh[32];
  long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int v = (i < n) ? in[i] : 0;
  int s = block_incl_scan(v, sh);
  if (threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = s;
}

// exclusive scan of the nb block sums in place, total at sums[nb]: one CTA of
// SCAN_BLOCK threads walks them in chunks with a running carry
__global__ void k_scan_sums(long long* sums, int nb) {
  __shared__ long long sh[SCAN_BLOCK / 32];
  __shared__ long long carry;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += SCAN_BLOCK) {
    int b = base + threadIdx.x;
    long long v = b < nb ? sums[b] : 0;
    long long s = v;
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane == 31) sh[w] = s;
    __syncthreads();
    if (w == 0) {
      long long t = sh[lane];
      for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      sh[lane] = t;
    }
    __syncthreads();
    if (w > 0) s += sh[w - 1];
    long long c = carry;
    if (b < nb) sums[b] = c + s - v;
    __syncthreads();
    if (threadIdx.x == SCAN_BLOCK - 1) carry = c + s;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_apply(const int* in, long long n, const long long* block_off, int* out) {
  __shared__ int sh[32];
  long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int v = (i < n) ? in[i] : 0;
  int s = block_incl_scan(v, sh);
  long long base = block_off[blockIdx.x];
  if (i < n) out[i] = (int)(base + s - v);
  if (i == n - 1) out[n] = (int)(base + s);
}

}  // namespace

namespace {

__global__ void k_take(const int* src, const int* idx, int n, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = src[idx[i]];
}

__global__ void k_any_negative(const int* v, long long n, int* flag) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && v[i] < 0) atomicExch(flag, 1);
}

}  // namespace

int take_ints(Batch& b, const int* src, const int* idx, int n, std::vector<int>& out) {
  out.assign(n, 0);
  if (n <= 0) return FAMS_OK;
  int* d = nullptr;
  FAMS_TRY(b.scratch((void**)&d, sizeof(int) * n));
  fams::note_launch(), k_take<<<grid_for(n, 256), 256, 0, b.stream>>>(src, idx, n, d);
  FAMS_CUDA(cudaMemcpyAsync(out.data(), d, sizeof(int) * n, cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  return FAMS_OK;
}

int any_negative(Batch& b, const int* v, long long n, bool* res) {
  *res = false;
  if (n <= 0) return FAMS_OK;
  int* d = nullptr;
  FAMS_TRY(b.scratch((void**)&d, sizeof(int)));
  FAMS_CUDA(cudaMemsetAsync(d, 0, sizeof(int), b.stream));
  fams::note_launch(), k_any_negative<<<grid_for(n, 256), 256, 0, b.stream>>>(v, n, d);
  int h = 0;
  FAMS_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  *res = h != 0;
  return FAMS_OK;
}

int fork_streams(Batch& b, int k, cudaStream_t* out) {
  if (!b.fk_ev[3]) FAMS_CUDA(cudaEventCreateWithFlags(&b.fk_ev[3], cudaEventDisableTiming));
  FAMS_CUDA(cudaEventRecord(b.fk_ev[3], b.stream));
  for (int i = 0; i < k; ++i) {
    if (!b.fk_st[i]) {
      FAMS_CUDA(cudaStreamCreateWithFlags(&b.fk_st[i], cudaStreamNonBlocking));
      FAMS_CUDA(cudaEventCreateWithFlags(&b.fk_ev[i], cudaEventDisableTiming));
    }
    FAMS_CUDA(cudaStreamWaitEvent(b.fk_st[i], b.fk_ev[3], 0));
    out[i] = b.fk_st[i];
  }
  return FAMS_OK;
}

int join_streams(Batch& b, int k) {
  for (int i = 0; i < k; ++i) {
    FAMS_CUDA(cudaEventRecord(b.fk_ev[i], b.fk_st[i]));
    FAMS_CUDA(cudaStreamWaitEvent(b.stream, b.fk_ev[i], 0));
  }
  return FAMS_OK;
}

int exclusive_scan(Batch& b, const int* in, int* out, long long n, long long* total) {
  if (n <= 0) {
    FAMS_CUDA(cudaMemsetAsync(out, 0, sizeof(int), b.stream));
    if (total) *total = 0;
    return FAMS_OK;
  }
  int nb = grid_for(n, SCAN_BLOCK);
  long long* sums = nullptr;
  FAMS_TRY(b.scratch((void**)&sums, sizeof(long long) * (nb + 1)));
  fams::note_launch(), k_scan_blocks<<<nb, SCAN_BLOCK, 0, b.stream>>>(in, n, sums);
  fams::note_launch(), k_scan_sums<<<1, SCAN_BLOCK, 0, b.stream>>>(sums, nb);
  fams::note_launch(), k_scan_apply<<<nb, SCAN_BLOCK, 0, b.stream>>>(in, n, sums, out);
  FAMS_CUDA(cudaGetLastError());
  long long tot = 0;
  FAMS_CUDA(cudaMemcpyAsync(&tot, sums + nb, sizeof(long long), cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  if (tot > 2147483647LL) {
    set_error("scan total exceeds the int32 index range");
    return FAMS_ECAPACITY;
  }
  if (total) *total = tot;
  return FAMS_OK;
}

namespace {

__global__ void k_count_cols(const int* col, long long nnz, int* cnt) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nnz) atomicAdd(&cnt[col[i]], 1);
}

__global__ void k_row_of(const int* rowptr, int nrows, int* rowof) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrows)
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) rowof[p] = r;
}

__global__ void k_place(const int* rowof, const int* col, const double* val, long long nnz,
                        const int* tptr, int* cursor, int* tcol, double* tval) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnz) return;
  int c = col[i];
  int pos = tptr[c] + atomicAdd(&cursor[c], 1);
  tcol[pos] = rowof[i];
  if (val) tval[pos] = val[i];
}

// bitonic sort of keys (and values) in place, m a power of two, one CTA
template <class K, class V>
__device__ void bitonic(K* sk, V* sv, int m) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          if ((sk[i] > sk[l]) == up) {
            K tk = sk[i]; sk[i] = sk[l]; sk[l] = tk;
            if (sv) { V tv = sv[i]; sv[i] = sv[l]; sv[l] = tv; }
          }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int SEG_TINY = 16;   // segments sorted by one thread in registers

// one thread per segment: segments of at most SEG_TINY entries are sorted in
// place by insertion; longer ones are listed for the CTA-per-segment sort
__global__ void k_seg_tiny(const int* ptr, int nseg, int* key, double* val, int* list, int* nlist) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int a = ptr[s], n = ptr[s + 1] - a;
  if (n <= 1) return;
  if (n > SEG_TINY) {
    list[atomicAdd(nlist, 1)] = s;
    return;
  }
  int k[SEG_TINY];
  double v[SEG_TINY];
  for (int i = 0; i < n; ++i) {
    int ki = key[a + i];
    double vi = val ? val[a + i] : 0.0;
    int j = i;
    while (j > 0 && k[j - 1] > ki) {
      k[j] = k[j - 1];
      v[j] = v[j - 1];
      --j;
    }
    k[j] = ki;
    v[j] = vi;
  }
  for (int i = 0; i < n; ++i) {
    key[a + i] = k[i];
    if (val) val[a + i] = v[i];
  }
}

// sort the listed segments with lo < length <= hi by key, one CTA per
// segment: in dynamic shared memory (gk null; room for the power of two above
// hi) or in a global scratch slice of `stride` keys (and values) per CTA
__global__ void k_seg_sort(const int* ptr, const int* list, int nseg, int* key, double* val,
                           int lo, int hi, int* gk, double* gv, long long stride) {
  extern __shared__ double dyn[];
  if ((int)blockIdx.x >= nseg) return;
  int s = list[blockIdx.x];
  int a = ptr[s], n = ptr[s + 1] - a;
  if (n <= lo || n > hi || n <= 1) return;
  int m = 1;
  while (m < n) m <<= 1;
  double* sv = gk ? (val ? gv + (long long)blockIdx.x * stride : nullptr) : (val ? dyn : nullptr);
  int* sk = gk ? gk + (long long)blockIdx.x * stride : (int*)(val ? dyn + m : dyn);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sk[i] = (i < n) ? key[a + i] : 0x7fffffff;
    if (sv) sv[i] = (i < n) ? val[a + i] : 0.0;
  }
  __syncthreads();
  bitonic(sk, sv, m);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    key[a + i] = sk[i];
    if (val) val[a + i] = sv[i];
  }
}

__global__ void k_seg_max(const int* ptr, int nseg, int* out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nseg) atomicMax(out, ptr[s + 1] - ptr[s]);
}

constexpr int SEG_SMALL = 1024;   // segments sorted with a small shared-memory footprint

}  // namespace

// sort each segment of `key` (and `val`) ascending: short segments in shared
// memory, longer ones in shared memory sized to the longest (up to what a CTA
// holds), the rest in global scratch.  `strict` is kept for the callers'
// intent: every segment is sorted.
int sort_segments(Batch& b, const int* ptr, int nseg, int* key, double* val, bool strict) {
  (void)strict;
  if (nseg <= 0) return FAMS_OK;
  int* dmax = nullptr;   // [0] longest segment, [1] listed segments
  int* list = nullptr;
  FAMS_TRY(b.scratch((void**)&dmax, sizeof(int) * 2));
  FAMS_TRY(b.scratch((void**)&list, sizeof(int) * nseg));
  FAMS_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int) * 2, b.stream));
  fams::note_launch(), k_seg_max<<<grid_for(nseg, 256), 256, 0, b.stream>>>(ptr, nseg, dmax);
  fams::note_launch(), k_seg_tiny<<<grid_for(nseg, 256), 256, 0, b.stream>>>(ptr, nseg, key, val,
                                                                           list, dmax + 1);
  int hm[2] = {0, 0};
  FAMS_CUDA(cudaMemcpyAsync(hm, dmax, sizeof(int) * 2, cudaMemcpyDeviceToHost, b.stream));
  FAMS_CUDA(cudaStreamSynchronize(b.stream));
  const int mx = hm[0], nl = hm[1];
  if (mx <= SEG_TINY || nl == 0) return FAMS_OK;
  const size_t per = sizeof(int) + (val ? sizeof(double) : 0);
  auto pow2 = [](int v) { int m = 1; while (m < v) m <<= 1; return m; };
  int max_smem = 0;
  FAMS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  FAMS_CUDA(cudaFuncSetAttribute(k_seg_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
  int small = std::min(mx, SEG_SMALL);
  fams::note_launch(), k_seg_sort<<<nl, 256, per * pow2(small), b.stream>>>(
      ptr, list, nl, key, val, SEG_TINY, SEG_SMALL, nullptr, nullptr, 0);
  if (mx > SEG_SMALL) {
    int cap = SEG_SMALL;
    while ((size_t)cap * 2 * per <= (size_t)max_smem && cap * 2 <= pow2(mx)) cap *= 2;
    if (cap > SEG_SMALL)
      fams::note_launch(), k_seg_sort<<<nl, 512, per * cap, b.stream>>>(
          ptr, list, nl, key, val, SEG_SMALL, cap, nullptr, nullptr, 0);
    if (mx > cap) {
      long long stride = pow2(mx);
      int *gk = nullptr;
      double* gv = nullptr;
      FAMS_TRY(b.scratch((void**)&gk, sizeof(int) * stride * (size_t)nl));
      if (val) FAMS_TRY(b.scratch((void**)&gv, sizeof(double) * stride * (size_t)nl));
      fams::note_launch(), k_seg_sort<<<nl, 1024, 0, b.stream>>>(ptr, list, nl, key, val, cap, 1 << 30,
                                                                gk, gv, stride);
    }
  }
  FAMS_CUDA(cudaGetLastError());
  return FAMS_OK;
}

int transpose(Batch& b, const int* rowptr, const int* col, const double* val, int nrows,
              int ncols, long long nnz, int** tptr, int** tcol, double** tval, bool keep) {
  int* cnt = nullptr;
  int* cursor = nullptr;
  int* rowof = nullptr;
  FAMS_TRY(b.scratch((void**)&cnt, sizeof(int) * (ncols + 1)));
  FAMS_TRY(b.scratch((void**)&cursor, sizeof(int) * (ncols + 1)));
  FAMS_TRY(b.scratch((void**)&rowof, sizeof(int) * (nnz + 1)));
  FAMS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (ncols + 1), b.stream));
  FAMS_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (ncols + 1), b.stream));
  auto alloc = [&](void** p, size_t bytes) { return keep ? b.alloc(p, bytes) : b.scratch(p, bytes); };
  FAMS_TRY(alloc((void**)tptr, sizeof(int) * (ncols + 1)));
  FAMS_TRY(alloc((void**)tcol, sizeof(int) * (nnz + 1)));
  if (tval) FAMS_TRY(alloc((void**)tval, sizeof(double) * (nnz + 1)));
  if (nnz > 0) {
    fams::note_launch(), k_count_cols<<<grid_for(nnz, 256), 256, 0, b.stream>>>(col, nnz, cnt);
    fams::note_launch(), k_row_of<<<grid_for(nrows, 256), 256, 0, b.stream>>>(rowptr, nrows, rowof);
  }
  FAMS_TRY(exclusive_scan(b, cnt, *tptr, ncols, nullptr));
  if (nnz > 0) {
    fams::note_launch(), k_place<<<grid_for(nnz, 256), 256, 0, b.stream>>>(rowof, col, val, nnz, *tptr, cursor, *tcol,
                                                      tval ? *tval : nullptr);
    FAMS_TRY(sort_segments(b, *tptr, ncols, *tcol, tval ? *tval : nullptr, true));
  }
  FAMS_CUDA(cudaGetLastError());
  return FAMS_OK;
}

}  // namespace fams
