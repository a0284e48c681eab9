// vd_bvh.cu -- input packing, Morton keys, radix sort and the power-augmented
// LBVH (App. A.1 "Input packing", App. A.2 "Power-augmented BVH"; the paper
// uses a third-party builder, this is a Karras-style binary radix tree over
// Morton-sorted sites, collapsed to leaves of at most `leaf_size` sites, with
// a per-node maximum weight for the culling test of Sec. 4.2.2).
#include "vd_internal.cuh"

namespace vd {

// ---------------------------------------------------------------- Morton keys

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  // spread the low 21 bits of v so that bit k lands on bit 3k (callers use
  // at most 20 bits per axis)
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ int find_set(const SetInfo* sets, int nsets, int i) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sets[mid].first <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Range of the weights of weighted sets (orderable-uint min / max).
__global__ void weight_range_kernel(const float* __restrict__ w, int n, const SetInfo* __restrict__ sets, int nsets,
                                    unsigned* __restrict__ wr) {
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int s = nsets > 1 ? find_set(sets, nsets, i) : 0;
    if (!sets[s].weighted || !isfinite(w[i])) continue;
    uint32_t o = f2o(w[i]);
    mn = min(mn, o);
    mx = max(mx, o);
  }
  mn = __reduce_min_sync(FULL, mn);
  mx = __reduce_max_sync(FULL, mx);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&wr[0], mn);
    atomicMax(&wr[1], mx);
  }
}

cudaError_t launch_weight_range(const float* w, int n, const SetInfo* sets, int nsets, unsigned* wr,
                                cudaStream_t s) {
  cudaMemsetAsync(wr, 0xff, sizeof(unsigned), s);
  cudaMemsetAsync(wr + 1, 0, sizeof(unsigned), s);
  if (!w) return cudaGetLastError();
  int blocks = min((n + 255) / 256, 1024);
  weight_range_kernel<<<blocks, 256, 0, s>>>(w, n, sets, nsets, wr);
  return cudaGetLastError();
}

// Weight stratum of a site (a performance device only; any partition
// gives the same cells): with o = w - w_min and O = w_max - w_min, bin 7
// holds o in (O/4, O], bin 6 (O/16, O/4], ... bin 0 everything below.
// Sorting by (bin, Morton) puts each stratum in its own subtrees, so a
// node's maximum weight -- the w_max of the node bound of Sec. 4.2.2 --
// is within a factor 4 of its sites' weights instead of the global maximum.
__device__ __forceinline__ uint32_t weight_bin(float w, float wmin, float wmax) {
  float O = wmax - wmin, o = w - wmin;
  if (!(O > 0.f) || !(o > 0.f)) return 0u;
  int k = (int)(0.5f * log2f(O / o));
  return (uint32_t)max(0, 7 - k);
}

__global__ void pack_keys_kernel(const float* __restrict__ xyz, const float* __restrict__ w, int n,
                                 const SetInfo* __restrict__ sets, int nsets, int set_shift, int bin_shift,
                                 const unsigned* __restrict__ wr, uint64_t* __restrict__ keys, int* __restrict__ vals,
                                 DevStatus* st) {
  const int bits = bin_shift / 3;
  const float scale = (float)(1u << bits);
  const float wmin = o2f(wr[0]), wmax = o2f(wr[1]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    int s = nsets > 1 ? find_set(sets, nsets, i) : 0;
    const SetInfo& S = sets[s];
    bool ok = isfinite(x) && isfinite(y) && isfinite(z);
    if (w && S.weighted) ok = ok && isfinite(w[i]);
    if (!ok) set_error(st, VD_ERR_INVALID_ARG);
    float c[3] = {x, y, z};
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float t = (c[k] - S.lo[k]) / (S.hi[k] - S.lo[k]);
      t = fminf(fmaxf(t, 0.0f), 1.0f);  // NaN -> 0 via fmaxf
      float v = floorf(t * scale);
      q[k] = (uint32_t)fminf(v, scale - 1.0f);
    }
    uint64_t code = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    uint32_t bin = (w && S.weighted && wr[0] <= wr[1]) ? weight_bin(w[i], wmin, wmax) : 0u;
    keys[i] = ((uint64_t)s << set_shift) | ((uint64_t)bin << bin_shift) | code;
    vals[i] = i;
  }
}

cudaError_t launch_pack_keys(const float* xyz, const float* w, int n, const SetInfo* sets, int nsets, int set_shift,
                             int bin_shift, const unsigned* wr, uint64_t* keys, int* vals, DevStatus* st,
                             cudaStream_t s) {
  int threads = 256;
  int blocks = (n + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  pack_keys_kernel<<<blocks, threads, 0, s>>>(xyz, w, n, sets, nsets, set_shift, bin_shift, wr, keys, vals, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
//
// Stable LSD radix sort of (uint64 key, int value) pairs, 8-bit digits.
// The array is cut into `nseg` contiguous segments, one per warp; every warp
// histograms its segment (upsweep), one block scans the digit-major
// histogram matrix, and every warp scatters its segment in order using
// __match_any_sync ranks within each 32-element chunk (downsweep).

constexpr int kSortWarpsPerBlock = 8;

__global__ void sort_upsweep(const uint64_t* __restrict__ keys, int n, int seg_len, int nseg, int shift,
                             unsigned* __restrict__ hist) {
  __shared__ unsigned h[kSortWarpsPerBlock][256];
  int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = lane; d < 256; d += 32) h[wib][d] = 0;
  __syncwarp();
  int seg = blockIdx.x * kSortWarpsPerBlock + wib;
  if (seg < nseg) {
    int b = seg * seg_len, e = min(n, b + seg_len);
    for (int i = b + lane; i < e; i += 32) {
      unsigned d = (unsigned)(keys[i] >> shift) & 255u;
      atomicAdd(&h[wib][d], 1u);
    }
  }
  __syncwarp();
  if (seg < nseg)
    for (int d = lane; d < 256; d += 32) hist[d * nseg + seg] = h[wib][d];
}

// exclusive scan of m entries with one block of 1024 threads
__global__ void sort_scan(unsigned* __restrict__ hist, int m) {
  __shared__ unsigned part[1024];
  int t = threadIdx.x;
  int per = (m + 1023) / 1024;
  int b = t * per, e = min(m, b + per);
  unsigned s = 0;
  for (int i = b; i < e; i++) s += hist[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned run = t ? part[t - 1] : 0u;
  for (int i = b; i < e; i++) {
    unsigned v = hist[i];
    hist[i] = run;
    run += v;
  }
}

__global__ void sort_downsweep(const uint64_t* __restrict__ keys, const int* __restrict__ vals, int n, int seg_len,
                               int nseg, int shift, const unsigned* __restrict__ hist,
                               uint64_t* __restrict__ keys_out, int* __restrict__ vals_out) {
  __shared__ unsigned base[kSortWarpsPerBlock][256];
  int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int seg = blockIdx.x * kSortWarpsPerBlock + wib;
  if (seg >= nseg) return;
  for (int d = lane; d < 256; d += 32) base[wib][d] = hist[d * nseg + seg];
  __syncwarp();
  int b = seg * seg_len, e = min(n, b + seg_len);
  unsigned lt = lanemask_lt();
  for (int c = b; c < e; c += 32) {
    int i = c + lane;
    bool act = i < e;
    uint64_t k = act ? keys[i] : ~0ull;
    int v = act ? vals[i] : 0;
    unsigned d = act ? ((unsigned)(k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(FULL, d);
    unsigned rank = __popc(peers & lt);
    unsigned pos = 0;
    if (act) pos = base[wib][d] + rank;
    __syncwarp();
    if (act) {
      keys_out[pos] = k;
      vals_out[pos] = v;
      // the highest lane of each peer group advances the digit's base
      if ((peers >> lane) == 1u) base[wib][d] += __popc(peers);
    }
    __syncwarp();
  }
}

cudaError_t radix_sort_pairs(uint64_t*& keys, uint64_t*& keys_alt, int*& vals, int*& vals_alt, unsigned* hist,
                             int n, int bits, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  int nseg = (n + 2047) / 2048;
  int maxseg = kSortBlocksMax * 2;  // hist holds 256 * kSortBlocksMax * 2 entries
  if (nseg > maxseg) nseg = maxseg;
  int seg_len = (n + nseg - 1) / nseg;
  seg_len = (seg_len + 31) & ~31;
  nseg = (n + seg_len - 1) / seg_len;
  int blocks = (nseg + kSortWarpsPerBlock - 1) / kSortWarpsPerBlock;
  for (int shift = 0; shift < bits; shift += 8) {
    sort_upsweep<<<blocks, 32 * kSortWarpsPerBlock, 0, s>>>(keys, n, seg_len, nseg, shift, hist);
    sort_scan<<<1, 1024, 0, s>>>(hist, 256 * nseg);
    sort_downsweep<<<blocks, 32 * kSortWarpsPerBlock, 0, s>>>(keys, vals, n, seg_len, nseg, shift, hist,
                                                              keys_alt, vals_alt);
    uint64_t* tk = keys;
    keys = keys_alt;
    keys_alt = tk;
    int* tv = vals;
    vals = vals_alt;
    vals_alt = tv;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- packed sorted sites

__global__ void gather_sites_kernel(const float* __restrict__ xyz, const float* __restrict__ w,
                                    const int* __restrict__ perm, int n, const SetInfo* __restrict__ sets,
                                    const uint64_t* __restrict__ keys, int set_shift, int nsets,
                                    float4* __restrict__ sites) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int i = perm[k];
    int s = nsets > 1 ? (int)(keys[k] >> set_shift) : 0;
    float wi = (w && sets[s].weighted) ? w[i] : 0.0f;
    sites[k] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], wi);
  }
}

cudaError_t launch_gather_sites(const float* xyz, const float* w, const int* perm, int n, const SetInfo* sets,
                                const uint64_t* keys, int set_shift, int nsets, float4* sites, cudaStream_t s) {
  int threads = 256;
  int blocks = min((n + threads - 1) / threads, 4096);
  gather_sites_kernel<<<blocks, threads, 0, s>>>(xyz, w, perm, n, sets, keys, set_shift, nsets, sites);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- duplicates
// Sites at exactly the same position share a Morton key and are adjacent
// after the sort. Among them the larger weight, then the lower original
// index, keeps its cell; every other one has an empty cell, and its
// half-space is implied by the winner's, so it is never a candidate.
__global__ void mark_losers_kernel(const uint64_t* __restrict__ keys, const float4* __restrict__ sites,
                                   const int* __restrict__ perm, int n, unsigned char* __restrict__ loser) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint64_t key = keys[k];
    float4 p = sites[k];
    bool lose = false;
    for (int dir = -1; dir <= 1 && !lose; dir += 2)
      for (int m = k + dir; m >= 0 && m < n && keys[m] == key && !lose; m += dir) {
        float4 q = sites[m];
        if (q.x == p.x && q.y == p.y && q.z == p.z)
          lose = q.w > p.w || (q.w == p.w && perm[m] < perm[k]);
      }
    loser[k] = lose ? 1 : 0;
  }
}

cudaError_t launch_mark_losers(const uint64_t* keys, const float4* sites, const int* perm, int n,
                               unsigned char* loser, cudaStream_t s) {
  int blocks = min((n + 255) / 256, 4096);
  mark_losers_kernel<<<blocks, 256, 0, s>>>(keys, sites, perm, n, loser);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Karras radix tree

__device__ __forceinline__ int common_prefix(const uint64_t* keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = keys[i], b = keys[j];
  if (a != b) return __clzll((long long)(a ^ b));
  return 64 + __clz(i ^ j);
}

// Internal node i of the binary radix tree over n sorted keys (ties broken
// by position). Children: internal index >= 0, or -1-site for a single site.
__global__ void karras_kernel(const uint64_t* __restrict__ keys, int n, int* __restrict__ left,
                              int* __restrict__ right, int* __restrict__ parent, int2* __restrict__ range) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int dplus = common_prefix(keys, n, i, i + 1), dminus = common_prefix(keys, n, i, i - 1);
  int d = dplus > dminus ? 1 : -1;
  int dmin = min(dplus, dminus);
  int lmax = 2;
  while (common_prefix(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (common_prefix(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = common_prefix(keys, n, i, j);
  int s = 0;
  int t = l;
  do {
    t = (t + 1) >> 1;
    if (common_prefix(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int gamma = i + s * d + min(d, 0);
  int lo = min(i, j), hi = max(i, j);
  int lc = (lo == gamma) ? (-1 - gamma) : gamma;
  int rc = (hi == gamma + 1) ? (-1 - (gamma + 1)) : (gamma + 1);
  left[i] = lc;
  right[i] = rc;
  range[i] = make_int2(lo, hi);
  // parent array: internal nodes at [0, n-1), sites at [n-1, 2n-1)
  parent[lc >= 0 ? lc : (n - 1) + (-1 - lc)] = i;
  parent[rc >= 0 ? rc : (n - 1) + (-1 - rc)] = i;
  if (i == 0) parent[0] = -1;
}

__device__ __forceinline__ void child_box(int c, const float4* sites, const float4* box_lo, const float4* box_hi,
                                          float4& lo, float4& hi) {
  if (c < 0) {
    float4 p = sites[-1 - c];
    lo = p;
    hi = make_float4(p.x, p.y, p.z, 0.0f);
  } else {
    lo = __ldcg(&box_lo[c]);
    hi = __ldcg(&box_hi[c]);
  }
}

// Bottom-up AABB + max-weight refit: the second visitor of a node merges
// its two children and walks on (no spinning on other threads).
__global__ void refit_kernel(const float4* __restrict__ sites, const int* __restrict__ left,
                             const int* __restrict__ right, const int* __restrict__ parent, int* visit,
                             float4* box_lo, float4* box_hi, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int p = parent[(n - 1) + k];
  while (p >= 0) {
    __threadfence();
    if (atomicAdd(&visit[p], 1) == 0) return;
    __threadfence();
    float4 a0, a1, b0, b1;
    child_box(left[p], sites, box_lo, box_hi, a0, a1);
    child_box(right[p], sites, box_lo, box_hi, b0, b1);
    float4 lo = make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), fmaxf(a0.w, b0.w));
    float4 hi = make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), fmaxf(a1.z, b1.z), 0.0f);
    __stcg(&box_lo[p], lo);
    __stcg(&box_hi[p], hi);
    p = parent[p];
  }
}

// Traversal record of internal node i: both children's boxes, max weights
// and references (64 bytes, read by four lanes with one float4 each).
__global__ void emit_nodes_kernel(const float4* __restrict__ sites, const int* __restrict__ left,
                                  const int* __restrict__ right, const int2* __restrict__ range,
                                  const float4* __restrict__ box_lo, const float4* __restrict__ box_hi, int n,
                                  int leaf_size, float4* __restrict__ nodes) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
#pragma unroll
  for (int c = 0; c < 2; c++) {
    int ch = c == 0 ? left[i] : right[i];
    float4 lo, hi;
    int ref;
    if (ch < 0) {
      float4 p = sites[-1 - ch];
      lo = p;
      hi = make_float4(p.x, p.y, p.z, 0.0f);
      ref = make_leaf_ref(-1 - ch, 1);
    } else {
      lo = box_lo[ch];
      hi = box_hi[ch];
      int2 r = range[ch];
      int cnt = r.y - r.x + 1;
      ref = cnt <= leaf_size ? make_leaf_ref(r.x, cnt) : ch;
    }
    hi.w = __int_as_float(ref);
    nodes[4 * i + 2 * c] = lo;
    nodes[4 * i + 2 * c + 1] = hi;
  }
}

// Root reference of every set: the node whose range is exactly the set.
__global__ void set_roots_kernel(SetInfo* sets, int nsets, const int2* __restrict__ range, int n, int leaf_size,
                                 DevStatus* st) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsets) return;
  int f = sets[s].first, c = sets[s].count;
  if (c <= 0) {
    sets[s].root = 0;
    return;
  }
  if (c <= leaf_size) {
    sets[s].root = make_leaf_ref(f, c);
    return;
  }
  int l = f + c - 1;
  int2 r;
  if (f < n - 1) {
    r = range[f];
    if (r.x == f && r.y == l) {
      sets[s].root = f;
      return;
    }
  }
  if (l < n - 1) {
    r = range[l];
    if (r.x == f && r.y == l) {
      sets[s].root = l;
      return;
    }
  }
  sets[s].root = 0;
  set_error(st, VD_ERR_INVALID_ARG);
}

cudaError_t launch_build_bvh(const uint64_t* keys, const float4* sites, int n, int leaf_size, BvhBuffers& b,
                             SetInfo* sets, int nsets, DevStatus* st, cudaStream_t s) {
  int threads = 256;
  if (n >= 2) {
    int blocks = (n - 1 + threads - 1) / threads;
    karras_kernel<<<blocks, threads, 0, s>>>(keys, n, b.left, b.right, b.parent, b.range);
    cudaMemsetAsync(b.visit, 0, sizeof(int) * (size_t)(n - 1), s);
    refit_kernel<<<(n + threads - 1) / threads, threads, 0, s>>>(sites, b.left, b.right, b.parent, b.visit,
                                                                  b.box_lo, b.box_hi, n);
    emit_nodes_kernel<<<blocks, threads, 0, s>>>(sites, b.left, b.right, b.range, b.box_lo, b.box_hi, n, leaf_size,
                                                 b.nodes);
  }
  set_roots_kernel<<<(nsets + 127) / 128, 128, 0, s>>>(sets, nsets, b.range, n, leaf_size, st);
  return cudaGetLastError();
}

}  // namespace vd
