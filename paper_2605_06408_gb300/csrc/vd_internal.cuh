// vd_internal.cuh -- device-side types and helpers shared by libvd's kernels.
//
// Coordinates inside a cell are local to its site (x~ = x - p_i). A plane is
// stored normalised: unit outward normal n^, offset b^ = signed distance of
// the plane from p_i (the d_ij of Eq. 2 for site planes), and e = an upper
// bound on |b^ - b^_exact| plus the rounding of one sign test against it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "vd.h"

namespace vd {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- limits
constexpr int kMaxLeaf = 32;            // leaf sizes 1..32 (one site per lane)
constexpr int kMaxSites = 1 << 26;      // leaf refs pack the first site in 26 bits
constexpr int kMaxSets = 1024;
constexpr int kBigWarpsPerBlock = 8;  // large-cell path: blocks of this many warps,
constexpr int kBigBlocksPerSm = 2;     // this many per SM (one arena per warp)
constexpr uint32_t kEmptyTri = 0xffffffffu;
#ifndef VD_KNN
#define VD_KNN 8
#endif
constexpr int kKnn = VD_KNN;          // sites of the KNN warm start (App. A.6)
constexpr int kKnnLeaf = -1;          // traversal reference of a cell's KNN list (no real leaf has it)

// Leaf references: bit 31 set, bits 26..30 = count-1, bits 0..25 = first.
__host__ __device__ inline int make_leaf_ref(int first, int count) {
  return (int)(0x80000000u | ((uint32_t)(count - 1) << 26) | (uint32_t)first);
}
__host__ __device__ inline bool ref_is_leaf(int ref) { return ref < 0; }
__host__ __device__ inline int leaf_first(int ref) { return (int)((uint32_t)ref & 0x03ffffffu); }
__host__ __device__ inline int leaf_count(int ref) { return (int)(((uint32_t)ref >> 26) & 31u) + 1; }

// ---------------------------------------------------------------- status
struct DevStatus {
  int error;
  int ovf_count;   // cells queued for the large-capacity pass
  long long nnz;
  long long empty_cells;
  long long overflow_cells;
  long long failed_cells;
  long long fp64_fallbacks;
  long long fp64_ambiguous;
  long long candidates;
  long long clips;
  long long nodes;
  long long vertex_tests;
  long long new_vertices;
  long long pool_used;  // ints of the large-cell neighbour pool in use
  long long nverts;     // vertices of the last mesh output
  long long refined_vertices;
  long long refined_volumes;
  long long ovf_reason[4];  // queue, vertices, planes, neighbours
  long long btape_used;     // bytes of the large-cell tape in use
  // counters of the large-cell pass (the fields above count the main pass)
  long long large_candidates;
  long long large_clips;
  long long large_nodes;
  long long large_vtests;
  long long large_newv;
  long long btape_records;   // large-cell polytopes written to the large-cell tape
  long long btape_restored;  // ... restored from it by the last adjoint
  int amb_count;             // cells with an FP64 sign test left inside its bound
  int amb_pad;
};

// Record cell `orig` (original index) as one whose construction took an FP64
// sign that was still inside its error bound.
__device__ inline void record_ambiguous(DevStatus* st, int* list, int cap, int orig) {
  const int k = atomicAdd(&st->amb_count, 1);
  if (k < cap) list[k] = orig;
}

__device__ inline void set_error(DevStatus* st, int code) { atomicCAS(&st->error, 0, code); }

// Per-set data of a (batched) build. Single builds use one set.
struct SetInfo {
  float lo[3], hi[3];
  int first;      // first site (original and sorted index space coincide per set)
  int count;
  int root;       // root reference (internal node index or leaf ref)
  int weighted;
};

// ---------------------------------------------------------------- numerics
template <typename T>
struct Num;
template <>
struct Num<float> {
  static constexpr float u = 5.9604644775390625e-8f;  // 2^-24
};
template <>
struct Num<double> {
  static constexpr double u = 1.1102230246251565e-16;  // 2^-53
};

template <typename T>
struct PlaneT {
  T nx, ny, nz, b, e;
};

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProduct):
// a + b = s + err and a * a = p + err exactly in floating point.
template <typename T>
__device__ __forceinline__ T two_sum_err(T a, T b, T s) {
  T bb = s - a;
  return (a - (s - bb)) + (b - bb);
}

// Radical plane of site q (weight wj) in the frame of site p (weight wi):
// n.x~ <= (|n|^2 + wi - wj)/2 with n = q - p (Eq. 1), normalised so that b
// is the power distance d_ij of Eq. 2. The offset is formed in compensated
// (float-float) arithmetic: each n_k = s_k + e_k exactly, s_k^2 = h_k + l_k
// exactly, the large terms are summed with TwoSum and the small ones added
// once, so 2b = |n|^2 + wi - wj carries a single rounding (u |2b|) plus
// terms of order u^2 (|n|^2 + |wi| + |wj|). With 1/|n| and the normal good
// to a few u, |b - b_exact| <= 6u|b| + 64u^2 (|n|^2 + |wi| + |wj|)/|n|;
// 10u|b| covers that and the 3u|b| of one fused sign test, so the bound
// scales with the plane's distance from p, not with |q - p|.
template <typename T>
__device__ __forceinline__ PlaneT<T> site_plane(T px, T py, T pz, T wi, T qx, T qy, T qz, T wj) {
  const T u = Num<T>::u;
  T sx = qx - px, sy = qy - py, sz = qz - pz;
  T ex = two_sum_err(qx, -px, sx), ey = two_sum_err(qy, -py, sy), ez = two_sum_err(qz, -pz, sz);
  T hx = sx * sx, hy = sy * sy, hz = sz * sz;
  T small = fma(sx, sx, -hx) + fma(sy, sy, -hy) + fma(sz, sz, -hz);
  small += fma(T(2) * sx, ex, ex * ex) + fma(T(2) * sy, ey, ey * ey) + fma(T(2) * sz, ez, ez * ez);
  T h1 = hx + hy;
  T c = two_sum_err(hx, hy, h1);
  T h2 = h1 + hz;
  c += two_sum_err(h1, hz, h2);
  T d = wi - wj;
  T cd = two_sum_err(wi, -wj, d);
  T A = h2 + d;
  T ca = two_sum_err(h2, d, A);
  T twob = A + (((ca + c) + small) + cd);
  T nn = h2 + (c + small);
  T r = T(1) / sqrt(nn);
  PlaneT<T> P;
  P.nx = fma(ex, r, sx * r);
  P.ny = fma(ey, r, sy * r);
  P.nz = fma(ez, r, sz * r);
  P.b = T(0.5) * twob * r;
  P.e = T(10) * u * fabs(P.b) + T(64) * u * u * (nn + fabs(wi) + fabs(wj)) * r;
  return P;
}

// Box face f (0:+x 1:-x 2:+y 3:-y 4:+z 5:-z) in the frame of p.
template <typename T>
__device__ __forceinline__ PlaneT<T> box_plane(int f, T px, T py, T pz, const float* lo, const float* hi) {
  const T u = Num<T>::u;
  int ax = f >> 1;
  T pc = ax == 0 ? px : (ax == 1 ? py : pz);
  PlaneT<T> P;
  P.nx = P.ny = P.nz = T(0);
  T s = (f & 1) ? T(-1) : T(1);
  if (ax == 0) P.nx = s;
  if (ax == 1) P.ny = s;
  if (ax == 2) P.nz = s;
  P.b = (f & 1) ? (pc - T(lo[ax])) : (T(hi[ax]) - pc);
  P.e = T(5) * u * fabs(P.b);
  return P;
}

// Vertex of planes (A, B, C) with det(nA, nB, nC) > 0 (orientation
// invariant), by Cramer's rule, and a bound e on |x - x_exact|_2 plus the
// rounding of a later sign test n^.x - b (first-order perturbation of the
// 3x3 system: |N^-1| <= sqrt(3)/W for unit normals, normal entries off by
// at most 8u, offsets by A.e etc.). e = inf when W is too small for the
// first-order bound to hold.
template <typename T>
__device__ __forceinline__ void vertex3(const PlaneT<T>& A, const PlaneT<T>& B, const PlaneT<T>& C, T& x, T& y,
                                        T& z, T& e) {
  const T u = Num<T>::u;
  const T epsn = T(8) * u;
  T c1x = fma(B.ny, C.nz, -B.nz * C.ny), c1y = fma(B.nz, C.nx, -B.nx * C.nz), c1z = fma(B.nx, C.ny, -B.ny * C.nx);
  T c2x = fma(C.ny, A.nz, -C.nz * A.ny), c2y = fma(C.nz, A.nx, -C.nx * A.nz), c2z = fma(C.nx, A.ny, -C.ny * A.nx);
  T c3x = fma(A.ny, B.nz, -A.nz * B.ny), c3y = fma(A.nz, B.nx, -A.nx * B.nz), c3z = fma(A.nx, B.ny, -A.ny * B.nx);
  T W = fma(A.nx, c1x, fma(A.ny, c1y, A.nz * c1z));
  T iw = T(1) / W;
  x = fma(A.b, c1x, fma(B.b, c2x, C.b * c3x)) * iw;
  y = fma(A.b, c1y, fma(B.b, c2y, C.b * c3y)) * iw;
  z = fma(A.b, c1z, fma(B.b, c2z, C.b * c3z)) * iw;
  T x1 = fabs(x) + fabs(y) + fabs(z);
  if (!(W > T(1024) * u) || !(x1 < T(1e30))) {
    e = T(INFINITY);
  } else {
    T ep = (T(1.75) * (A.e + B.e + C.e) + (T(5.25) * epsn + T(9) * u) * x1 +
            T(6) * u * (fabs(A.b) + fabs(B.b) + fabs(C.b))) * iw + u * x1;
    e = T(1.1) * ep + (epsn + T(3) * u) * x1;
  }
}

// Sign test value s = n^.x - b (>0: outside) and whether it is certain.
template <typename T>
__device__ __forceinline__ T side(const PlaneT<T>& H, T x, T y, T z) {
  return fma(H.nx, x, fma(H.ny, y, fma(H.nz, z, -H.b)));
}

template <typename T>
__device__ __forceinline__ bool ambiguous(T s, T ev, T eh) {
  return fabs(s) <= (ev + eh) * (T(1) + T(4) * Num<T>::u);
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
// monotone map float -> uint32 (for redux.sync min/max)
__device__ __forceinline__ uint32_t f2o(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(u);
}
__device__ __forceinline__ float warp_minf(float v) { return o2f(__reduce_min_sync(FULL, f2o(v))); }
__device__ __forceinline__ float warp_maxf(float v) { return o2f(__reduce_max_sync(FULL, f2o(v))); }
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ---------------------------------------------------------------- host-side launchers
struct BvhBuffers {
  // sorting
  uint64_t* keys;
  uint64_t* keys_alt;
  int* vals;
  int* vals_alt;
  unsigned* hist;      // [256 * 2 * kSortBlocksMax]
  // Karras tree
  int* left;
  int* right;
  int* parent;         // [2n-1]: parents of internal nodes then of sites
  int2* range;
  int* visit;
  float4* box_lo;      // per internal node: lo.xyz, maxw
  float4* box_hi;      // hi.xyz
  float4* nodes;       // [n-1][4] traversal records
};

// Tape of the forward's cells for the adjoint: one record of kTapeStride
// bytes per sorted site: int4 header (vertex count, face count; vertex count
// -1 = no record, the adjoint re-clips), kTapeV float4 vertices (local
// position, plane triplet bits in w, indices into the record's faces), kTapeF
// face ids (sorted site index, or -1-f for box face f).
constexpr int kTapeV = 48;
constexpr int kTapeF = 32;
constexpr int kTapeStride = 1024;
constexpr int kTapeVOff = 16;
constexpr int kTapeFOff = kTapeVOff + 16 * kTapeV;

struct CellBuffers {
  const float4* sites;   // sorted packed sites
  const unsigned char* loser;  // sorted index: an exact duplicate site beats it
  const int* perm;       // sorted -> original index
  const float4* nodes;
  const uint64_t* keys;  // sorted keys (set id in the top bits)
  const SetInfo* sets;
  int nsets;
  int set_shift;
  int n;
  int* counts;           // [n] by original index
  int* scratch;          // [n * stride]
  int stride;
  int* pool;             // neighbour lists of large cells
  long long pool_cap;
  char* arena;           // per-warp arenas of the large-cell path
  int* ovf_list;         // [ovf_cap] sorted indices of overflowed cells
  int ovf_cap;
  int* ovf_slot;         // [n] by original index: offset in `pool` or -1
  float* vol;
  float* cen;
  int* work;             // [2] work counters (main pass, overflow pass)
  DevStatus* st;
  char* tape;            // [n * kTapeStride] or nullptr (no tape this build)
  int* stall;            // test hook: armed token (one helping group is never counted), or nullptr
  vd_config cfg;
  char* btape;           // large-cell tape (polytopes of cells past the register path), or nullptr
  long long btape_cap;   // its bytes
  int* amb_list;         // [amb_cap] original ids of cells with an FP64-ambiguous sign test
  int amb_cap;
  int cell_begin;        // the cells this build makes: sorted indices [cell_begin, cell_end)
  int cell_end;          //   (all of [0, n) unless the context is partitioned)
  const int* knn;        // [n * kKnn] nearest sites (sorted indices, -1 = none) for warm_start = 2
};

constexpr int kSortThreads = 512;
constexpr int kSortBlocksMax = 1024;

struct BackBuffers {
  CellBuffers c;
  const int* inv_perm;  // original -> sorted index
  const float* gvol;
  const float* gcen;
  float* gp;
  float* gw;
  int* list;            // cells that overflowed the small variant
  int* list_count;
  int list_cap;
  int* work;            // [2]
  const char* tape;     // the forward's tape, or nullptr (re-clip every cell)
  // mesh output and vertex gradients
  int mode;              // 0: gradients; 1: vertex count per cell; 2: vertex output
  int* vcount;           // [n] by original index (mode 1)
  const int32_t* voff;   // [n+1] vertex offsets (mode 2; mode 0 with gvert)
  float* vout;           // [3 vcap] world positions (mode 2)
  int32_t* vsites;       // [3 vcap] the other three defining sites (mode 2)
  long long vcap;        // (mode 2)
  const float* gvert;    // [3 V] gradient per vertex in mesh order, or nullptr
};

cudaError_t launch_weight_range(const float* w, int n, const SetInfo* sets, int nsets, unsigned* wr,
                                cudaStream_t s);
cudaError_t launch_pack_keys(const float* xyz, const float* w, int n, const SetInfo* sets, int nsets, int set_shift,
                             int bin_shift, const unsigned* wr, uint64_t* keys, int* vals, DevStatus* st,
                             cudaStream_t s);
cudaError_t radix_sort_pairs(uint64_t*& keys, uint64_t*& keys_alt, int*& vals, int*& vals_alt, unsigned* hist,
                             int n, int bits, cudaStream_t s);
cudaError_t launch_gather_sites(const float* xyz, const float* w, const int* perm, int n, const SetInfo* sets,
                                const uint64_t* keys, int set_shift, int nsets, float4* sites, cudaStream_t s);
cudaError_t launch_build_bvh(const uint64_t* keys, const float4* sites, int n, int leaf_size, BvhBuffers& b,
                             SetInfo* sets, int nsets, DevStatus* st, cudaStream_t s);
cudaError_t launch_cells(const CellBuffers& c, int num_sms, cudaStream_t s, const std::function<void()>& between);
cudaError_t launch_cells_thread(const CellBuffers& c, int num_sms, cudaStream_t s);
cudaError_t launch_knn(const CellBuffers& c, int* knn, cudaStream_t s);
cudaError_t launch_csr(const CellBuffers& c, int32_t* offsets, int32_t* neighbors, int64_t cap, int64_t* nnz_out,
                       long long* block_sums, int32_t* user_status, bool recount, cudaStream_t s);
cudaError_t launch_backward(const BackBuffers& b, int num_sms, cudaStream_t s);
cudaError_t launch_scan(const int* counts, int n, int32_t* offsets, long long* block_sums, long long* total,
                        DevStatus* st, cudaStream_t s);
cudaError_t launch_mesh_finish(const DevStatus* st, int64_t* nverts_out, int32_t* user_status, cudaStream_t s);
cudaError_t launch_inverse_perm(const int* perm, int n, int* inv, cudaStream_t s);
cudaError_t launch_mark_losers(const uint64_t* keys, const float4* sites, const int* perm, int n,
                               unsigned char* loser, cudaStream_t s);

}  // namespace vd
