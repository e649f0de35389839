// Device-wide helpers used by the setup phases: exclusive scan and a CSR
// transpose whose segments come out sorted (deterministic, no atomics in the
// final order).
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

__global__ void k_scan_sums(long long* sums, int nb) {
  // single thread: block counts are small (n / 1024)
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long acc = 0;
    for (int b = 0; b < nb; ++b) {
      long long t = sums[b];
      sums[b] = acc;
      acc += t;
    }
    sums[nb] = acc;
  }
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
  fams::note_launch(), k_scan_sums<<<1, 32, 0, b.stream>>>(sums, nb);
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

// sort each segment by key (one CTA per segment, in shared memory)
constexpr int SEG_SORT_MAX = 4096;
__global__ void k_seg_sort(const int* ptr, int nseg, int* key, double* val, int* err,
                           int strict) {
  __shared__ int sk[SEG_SORT_MAX];
  __shared__ double sv[SEG_SORT_MAX];
  int s = blockIdx.x;
  if (s >= nseg) return;
  int a = ptr[s], n = ptr[s + 1] - a;
  if (n <= 1) return;
  if (n > SEG_SORT_MAX) {
    if (strict && threadIdx.x == 0) atomicCAS(err, 0, DERR_CAPACITY);
    return;
  }
  int m = 1;
  while (m < n) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sk[i] = (i < n) ? key[a + i] : 0x7fffffff;
    sv[i] = (i < n && val) ? val[a + i] : 0.0;
  }
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          if ((sk[i] > sk[l]) == up) {
            int tk = sk[i]; sk[i] = sk[l]; sk[l] = tk;
            double tv = sv[i]; sv[i] = sv[l]; sv[l] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    key[a + i] = sk[i];
    if (val) val[a + i] = sv[i];
  }
}

}  // namespace

int sort_segments(Batch& b, const int* ptr, int nseg, int* key, double* val, bool strict) {
  if (nseg <= 0) return FAMS_OK;
  fams::note_launch(), k_seg_sort<<<nseg, 256, 0, b.stream>>>(ptr, nseg, key, val, b.d_err, strict ? 1 : 0);
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
