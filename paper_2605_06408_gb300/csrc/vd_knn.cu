// vd_knn.cu -- the K nearest sites of every site, by a query on the LBVH:
// the input of the KNN warm start of App. A.6 (vd_config.warm_start = 2),
// where each cell is first clipped by the planes of its K = 8 nearest
// sites, so that the directional bounds are tight from the first node test
// of the traversal on.
//
// One thread per site (the query is short and independent per site): a
// depth-first descent of the site's set's subtree, nearer child first, with
// an explicit stack of (node, squared box distance); a node is skipped once
// its box is farther than the current K-th nearest site. The K best stay
// sorted in registers. Any K sites give a valid warm start (clipping by any
// site's plane keeps the exact cell), so a stack that runs out of room only
// makes the list approximate, never wrong.
#include "vd_internal.cuh"

namespace vd {

namespace {

constexpr int kKnnStack = 64;

// squared distance from p to the box [lo, hi] (0 inside)
__device__ __forceinline__ float box_d2(const float4& p, const float4& lo, const float4& hi) {
  const float dx = fmaxf(fmaxf(lo.x - p.x, p.x - hi.x), 0.0f);
  const float dy = fmaxf(fmaxf(lo.y - p.y, p.y - hi.y), 0.0f);
  const float dz = fmaxf(fmaxf(lo.z - p.z, p.z - hi.z), 0.0f);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

__global__ void __launch_bounds__(128) knn_kernel(const float4* __restrict__ sites, const float4* __restrict__ nodes,
                                                  const SetInfo* __restrict__ sets, int nsets,
                                                  const uint64_t* __restrict__ keys, int set_shift,
                                                  const unsigned char* __restrict__ loser, int n, int begin,
                                                  int end, int* __restrict__ knn) {
  const int si = begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (si >= end) return;
  const float4 p = sites[si];
  const int set = nsets > 1 ? (int)(keys[si] >> set_shift) : 0;
  float bd[kKnn];
  int bi[kKnn];
#pragma unroll
  for (int k = 0; k < kKnn; k++) {
    bd[k] = INFINITY;
    bi[k] = -1;
  }
  int sref[kKnnStack];
  float sd[kKnnStack];
  int top = 0;
  sref[top] = sets[set].root;
  sd[top++] = 0.0f;
  while (top > 0) {
    --top;
    const int ref = sref[top];
    if (!(sd[top] < bd[kKnn - 1])) continue;  // farther than the K-th best by now
    if (ref_is_leaf(ref)) {
      const int f = leaf_first(ref), c = leaf_count(ref);
      for (int j = f; j < f + c; j++) {
        if (j == si || loser[j]) continue;
        const float4 q = sites[j];
        const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
        float cd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(cd < bd[kKnn - 1])) continue;
        int cj = j;
#pragma unroll
        for (int k = 0; k < kKnn; k++) {  // insert, keeping the list sorted
          if (cd < bd[k]) {
            const float td = bd[k];
            const int tj = bi[k];
            bd[k] = cd;
            bi[k] = cj;
            cd = td;
            cj = tj;
          }
        }
      }
      continue;
    }
    const float4* nd = nodes + 4 * (size_t)ref;
    const float4 l0 = nd[0], h0 = nd[1], l1 = nd[2], h1 = nd[3];
    float d0 = box_d2(p, l0, h0), d1 = box_d2(p, l1, h1);
    int r0 = __float_as_int(h0.w), r1 = __float_as_int(h1.w);
    if (d1 < d0) {  // child 0 becomes the nearer one
      const float td = d0;
      d0 = d1;
      d1 = td;
      const int tr = r0;
      r0 = r1;
      r1 = tr;
    }
    // the farther child below the nearer one on the stack: the nearer is
    // popped first
    if (d1 < bd[kKnn - 1] && top < kKnnStack) {
      sref[top] = r1;
      sd[top++] = d1;
    }
    if (d0 < bd[kKnn - 1] && top < kKnnStack) {
      sref[top] = r0;
      sd[top++] = d0;
    }
  }
#pragma unroll
  for (int k = 0; k < kKnn; k++) knn[(size_t)si * kKnn + k] = bi[k];
}

}  // namespace

cudaError_t launch_knn(const CellBuffers& c, int* knn, cudaStream_t s) {
  const int m = c.cell_end - c.cell_begin;
  if (m <= 0) return cudaSuccess;
  knn_kernel<<<(m + 127) / 128, 128, 0, s>>>(c.sites, c.nodes, c.sets, c.nsets, c.keys, c.set_shift, c.loser, c.n,
                                            c.cell_begin, c.cell_end, knn);
  return cudaGetLastError();
}

}  // namespace vd
