// vd_csr.cu -- neighbour counts -> CSR row offsets (exclusive prefix sum) ->
// compacted neighbour array. The paper states only that the full
// connectivity is produced (App. A.3); this is the count / scan / compact
// layout of it.
#include "vd_internal.cuh"

namespace vd {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// inclusive block scan of one value per thread (1024 threads)
__device__ __forceinline__ long long block_inclusive_scan(long long v, long long* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(FULL, w, o);
      if (lane >= o) w += t;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += warp_tot[wid - 1];
  return v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int* __restrict__ counts, int n,
                                                                   long long* __restrict__ bsum) {
  __shared__ long long wt[32];
  long long s = 0;
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
#pragma unroll
  for (int k = 0; k < kScanItems; k++)
    if (base + k < n) s += counts[base + k];
  s = block_inclusive_scan(s, wt);
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads) scan_bsum_kernel(long long* bsum, int nb, long long* total,
                                                                 DevStatus* st) {
  __shared__ long long wt[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    int i = b0 + threadIdx.x;
    long long v = i < nb ? bsum[i] : 0;
    long long inc = block_inclusive_scan(v, wt);
    long long c0 = carry;
    __syncthreads();
    if (i < nb) bsum[i] = c0 + inc - v;  // exclusive
    if (threadIdx.x == kScanThreads - 1) carry = c0 + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry;
    if (carry > 0x7fffffffLL) set_error(st, VD_ERR_TOO_LARGE);
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_write_kernel(const int* __restrict__ counts, int n,
                                                                  const long long* __restrict__ bsum,
                                                                  int* __restrict__ offsets,
                                                                  const long long* __restrict__ total) {
  __shared__ long long wt[32];
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int c[kScanItems];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    c[k] = base + k < n ? counts[base + k] : 0;
    s += c[k];
  }
  long long inc = block_inclusive_scan(s, wt);
  long long run = bsum[blockIdx.x] + inc - s;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) offsets[base + k] = (int)run;
    run += c[k];
  }
  if (base + kScanItems >= n && base < n) offsets[n] = (int)*total;
}

// one warp per row: copy the row's neighbours from its scratch row (or the
// large-cell pool)
__global__ void compact_kernel(const int* __restrict__ counts, const int* __restrict__ offsets,
                               const int* __restrict__ scratch, int stride, const int* __restrict__ pool,
                               const int* __restrict__ ovf_slot, int n, int* __restrict__ nbrs,
                               long long cap, const DevStatus* st) {
  long long nnz = st->nnz;
  if (nnz > cap || nnz > 0x7fffffffLL) return;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
    int cnt = counts[row];
    if (cnt <= 0) continue;
    int slot = ovf_slot[row];
    const int* src = slot >= 0 ? pool + slot : scratch + (size_t)row * stride;
    int* dst = nbrs + offsets[row];
    for (int k = lane; k < cnt; k += 32) dst[k] = src[k];
  }
}

__global__ void finish_status_kernel(DevStatus* st, long long cap, int64_t* nnz_out, int32_t* user_status) {
  long long nnz = st->nnz;
  if (nnz > cap)
    set_error(st, VD_ERR_CAPACITY);
  else
    atomicCAS(&st->error, VD_ERR_CAPACITY, 0);  // a re-copy into a large enough buffer
  if (nnz_out) *nnz_out = nnz;
  if (user_status) *user_status = st->error;
}

cudaError_t launch_csr(const CellBuffers& c, int32_t* offsets, int32_t* neighbors, int64_t cap, int64_t* nnz_out,
                       long long* block_sums, int32_t* user_status, bool recount, cudaStream_t s) {
  int n = c.n;
  int nb = (n + kScanTile - 1) / kScanTile;
  if (recount) {
    scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(c.counts, n, block_sums);
    scan_bsum_kernel<<<1, kScanThreads, 0, s>>>(block_sums, nb, &c.st->nnz, c.st);
    scan_write_kernel<<<nb, kScanThreads, 0, s>>>(c.counts, n, block_sums, offsets, &c.st->nnz);
  }
  if (neighbors && cap > 0) {
    int blocks = (n + 7) / 8;
    if (blocks > 65536) blocks = 65536;
    compact_kernel<<<blocks, 256, 0, s>>>(c.counts, offsets, c.scratch, c.stride, c.pool, c.ovf_slot, n,
                                          neighbors, neighbors ? cap : 0, c.st);
  }
  finish_status_kernel<<<1, 1, 0, s>>>(c.st, neighbors ? cap : 0x7fffffffffffffffLL, nnz_out, user_status);
  return cudaGetLastError();
}

__global__ void mesh_finish_kernel(const DevStatus* st, int64_t* nverts_out, int32_t* user_status) {
  if (nverts_out) *nverts_out = st->nverts;
  if (user_status) *user_status = st->error;
}

cudaError_t launch_mesh_finish(const DevStatus* st, int64_t* nverts_out, int32_t* user_status, cudaStream_t s) {
  mesh_finish_kernel<<<1, 1, 0, s>>>(st, nverts_out, user_status);
  return cudaGetLastError();
}

// Exclusive scan of n counts into offsets[n+1]; the total goes to *total.
cudaError_t launch_scan(const int* counts, int n, int32_t* offsets, long long* block_sums, long long* total,
                        DevStatus* st, cudaStream_t s) {
  int nb = (n + kScanTile - 1) / kScanTile;
  scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(counts, n, block_sums);
  scan_bsum_kernel<<<1, kScanThreads, 0, s>>>(block_sums, nb, total, st);
  scan_write_kernel<<<nb, kScanThreads, 0, s>>>(counts, n, block_sums, offsets, total);
  return cudaGetLastError();
}

}  // namespace vd
