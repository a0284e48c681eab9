// vd_clip.cuh -- the per-cell polytope held by one warp and its clipping
// step (Sec. 4.1, App. B), shared by the forward and the adjoint kernels.
//
// Vertices live in registers: VPL slots per lane, each with its position
// (local frame), an error bound and its plane triplet (a | b<<8 | c<<16,
// det(n_a, n_b, n_c) > 0). Planes live in shared memory. A clip by plane h
// classifies all vertices in parallel, collects the outside ones, and finds
// the boundary of the hole as the directed plane pairs (a,b) of outside
// vertices whose reverse pair (b,a) belongs to no other outside vertex;
// each becomes the new vertex (a,b,h). That is the polytope the paper's
// sequential walk around the hole produces, computed on 32 lanes at once.
//
// Predicates run in FP32; a sign test whose value lies within its error
// bound of zero is re-evaluated in FP64 from the original inputs.
#pragma once

#include "vd_internal.cuh"

namespace vd {

constexpr float kCullPad = 1e-5f;

template <int VPL, int PCAP>
struct WarpSmem {
  float4 pl[PCAP];   // n^x, n^y, n^z, b^ (local frame)
  float pe[PCAP];    // offset error bound per plane
  int pid[PCAP];     // sorted site index, or -1-f for box face f
  uint32_t otri[32 * VPL];
  float4 nvp[32 * VPL];
  uint32_t nvt[32 * VPL];
};

struct Counters {
  long long cand, clips, nodes, vtests, newv, fp64, fp64amb;
};

template <int VPL, int PCAP, int QPL>
struct Cell {
  static constexpr int VCAP = 32 * VPL;
  static constexpr int NPW = PCAP / 32;
  // vertices (per lane)
  float vx[VPL], vy[VPL], vz[VPL], ve[VPL];
  uint32_t vt[VPL];
  // best-first queue (per lane)
  float qlb[QPL];
  int qref[QPL];
  int qocc[QPL];  // occupied-octant bits | push sequence << 8; < 0 = empty
  // warp-uniform state
  float4 me;
  float lo[3], hi[3];  // the set's box
  float alo[3], ahi[3];
  int nv;
  uint32_t freem[NPW];
  int seq;
  bool dirty;
};

template <int VPL, int PCAP>
__device__ __forceinline__ PlaneT<float> load_plane(const WarpSmem<VPL, PCAP>& S, int k) {
  float4 t = S.pl[k];
  PlaneT<float> P;
  P.nx = t.x;
  P.ny = t.y;
  P.nz = t.z;
  P.b = t.w;
  P.e = S.pe[k];
  return P;
}

__device__ __forceinline__ PlaneT<double> plane64(int id, const float4& me, const float* lo, const float* hi,
                                                  const float4* __restrict__ sites) {
  if (id >= 0) {
    float4 q = sites[id];
    return site_plane<double>(me.x, me.y, me.z, me.w, q.x, q.y, q.z, q.w);
  }
  return box_plane<double>(-1 - id, me.x, me.y, me.z, lo, hi);
}

// FP64 re-evaluation of "vertex tri lies outside the plane of site hpid".
template <int VPL, int PCAP>
__device__ __noinline__ bool resolve64(const WarpSmem<VPL, PCAP>& S, uint32_t tri, int hpid, float4 me,
                                       const float* lo, const float* hi, const float4* __restrict__ sites,
                                       long long& amb) {
  PlaneT<double> A = plane64(S.pid[tri & 255u], me, lo, hi, sites);
  PlaneT<double> B = plane64(S.pid[(tri >> 8) & 255u], me, lo, hi, sites);
  PlaneT<double> C = plane64(S.pid[(tri >> 16) & 255u], me, lo, hi, sites);
  double x, y, z, e;
  vertex3<double>(A, B, C, x, y, z, e);
  PlaneT<double> H = plane64(hpid, me, lo, hi, sites);
  double s = side<double>(H, x, y, z);
  if (ambiguous<double>(s, e, H.e)) amb++;
  return s > 0.0;
}

// squared directional radius over the octants in `occ` (Sec. 4.2.1/4.2.2):
// the largest squared distance from the site to the cell-AABB corner that
// faces each occupied octant; cull_mode 1 takes every octant (isotropic).
__device__ __forceinline__ float dir_radius2(int occ, const float* alo, const float* ahi, int cull_mode) {
  float r2 = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    bool pos = cull_mode == 1 || ((occ >> (2 * k)) & 1);
    bool neg = cull_mode == 1 || ((occ >> (2 * k + 1)) & 1);
    float a = pos ? ahi[k] * ahi[k] : 0.0f;
    float b = neg ? alo[k] * alo[k] : 0.0f;
    r2 += fmaxf(a, b);
  }
  return r2;
}

template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ void recompute_aabb(Cell<VPL, PCAP, QPL>& c) {
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, em = 0.0f;
#pragma unroll
  for (int r = 0; r < VPL; r++)
    if (c.vt[r] != kEmptyTri) {
      mn[0] = fminf(mn[0], c.vx[r]);
      mn[1] = fminf(mn[1], c.vy[r]);
      mn[2] = fminf(mn[2], c.vz[r]);
      mx[0] = fmaxf(mx[0], c.vx[r]);
      mx[1] = fmaxf(mx[1], c.vy[r]);
      mx[2] = fmaxf(mx[2], c.vz[r]);
      em = fmaxf(em, c.ve[r]);
    }
  em = warp_maxf(em);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.alo[k] = warp_minf(mn[k]) - em;
    c.ahi[k] = warp_maxf(mx[k]) + em;
  }
}

// Test of one BVH child box [lo.xyz, hi.xyz] with maximum weight lo.w
// (Sec. 4.2.2): d = distance from the site to the box, lower bound of every
// d_ij in the box LB = d/2 + min(0, w_i - w_max)/(2d); culled iff LB exceeds
// the directional radius over the octants the box occupies. Returns keep;
// lb is a safe (padded) LB, key the best-first key LB - R.
__device__ __forceinline__ bool node_test(float4 lo, float4 hi, float4 me, const float* alo, const float* ahi,
                                          int cull_mode, float& lb, int& occ, float& key) {
  float rl[3] = {lo.x - me.x, lo.y - me.y, lo.z - me.z};
  float rh[3] = {hi.x - me.x, hi.y - me.y, hi.z - me.z};
  float d2 = 0.0f;
  occ = 0;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float dk = fmaxf(fmaxf(rl[k], -rh[k]), 0.0f);
    d2 = fmaf(dk, dk, d2);
    occ |= (rh[k] >= 0.0f ? 1 : 0) << (2 * k);
    occ |= (rl[k] <= 0.0f ? 1 : 0) << (2 * k + 1);
  }
  float R = sqrtf(dir_radius2(occ, alo, ahi, cull_mode));
  if (d2 == 0.0f) {
    lb = -INFINITY;
    key = -R;
    return true;
  }
  float d = sqrtf(d2);
  float c = fminf(0.0f, me.w - lo.w);
  lb = (d2 + c - kCullPad * (d2 + fabsf(me.w) + fabsf(lo.w))) / (2.0f * d);
  key = (d2 + c) / (2.0f * d) - R;
  if (cull_mode == 2) return true;
  return !(lb > R * (1.0f + kCullPad));
}

template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ bool queue_push(Cell<VPL, PCAP, QPL>& c, float lb, int ref, int occ) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int r = 0; r < QPL; r++) {
    unsigned fm = __ballot_sync(FULL, c.qocc[r] < 0);
    if (fm) {
      if (lane == (unsigned)(__ffs(fm) - 1)) {
        c.qlb[r] = lb;
        c.qref[r] = ref;
        c.qocc[r] = occ | (c.seq << 8);
      }
      c.seq++;
      return true;
    }
  }
  return false;
}

// Pop the most promising entry still valid under the current cell bounds
// (Alg. 1 backtracking: re-test with the shrunken radii; entries that now
// fail are discarded). Depth-first mode pops the newest entry.
template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ bool queue_pop(Cell<VPL, PCAP, QPL>& c, int cull_mode, int traversal, int& ref) {
  const unsigned lane = lane_id();
  uint32_t best = 0xffffffffu;
  int bslot = 0;
#pragma unroll
  for (int r = 0; r < QPL; r++) {
    if (c.qocc[r] >= 0) {
      float R = sqrtf(dir_radius2(c.qocc[r] & 63, c.alo, c.ahi, cull_mode));
      if (cull_mode != 2 && c.qlb[r] > R * (1.0f + kCullPad)) {
        c.qocc[r] = -1;
        continue;
      }
      uint32_t k = traversal == 0 ? f2o(c.qlb[r] - R) : (0xfffffffeu - (uint32_t)(c.qocc[r] >> 8));
      if (k < best) {
        best = k;
        bslot = r;
      }
    }
  }
  uint32_t mn = __reduce_min_sync(FULL, best);
  if (mn == 0xffffffffu) return false;
  int src = __ffs(__ballot_sync(FULL, best == mn)) - 1;
  int mine = 0;
#pragma unroll
  for (int r = 0; r < QPL; r++)
    if (r == bslot) mine = c.qref[r];
  ref = __shfl_sync(FULL, mine, src);
  if ((int)lane == src) {
#pragma unroll
    for (int r = 0; r < QPL; r++)
      if (r == bslot) c.qocc[r] = -1;
  }
  return true;
}

enum { CLIP_NONE = 0, CLIP_DONE = 1, CLIP_EMPTY = 2, CLIP_OVERFLOW = 3 };

// Clip the cell by plane H of site hpid (App. B "Clipping by a half-space").
template <int VPL, int PCAP, int QPL>
__device__ int clip_cell(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP>& S, const PlaneT<float>& H, int hpid,
                         const float4* __restrict__ sites, Counters& ct, bool counters) {
  constexpr int VCAP = Cell<VPL, PCAP, QPL>::VCAP;
  constexpr int NPW = Cell<VPL, PCAP, QPL>::NPW;
  const unsigned lane = lane_id(), lt = lanemask_lt();
  bool out[VPL];
  // step 1: classify every vertex
#pragma unroll
  for (int r = 0; r < VPL; r++) {
    out[r] = false;
    if (c.vt[r] != kEmptyTri) {
      float s = side<float>(H, c.vx[r], c.vy[r], c.vz[r]);
      out[r] = s > 0.0f;
      if (ambiguous<float>(s, c.ve[r], H.e)) {
        ct.fp64++;
        out[r] = resolve64(S, c.vt[r], hpid, c.me, c.lo, c.hi, sites, ct.fp64amb);
      }
    }
  }
  if (counters) ct.vtests += c.nv;
  uint32_t om[VPL];
  int k = 0;
#pragma unroll
  for (int r = 0; r < VPL; r++) {
    om[r] = __ballot_sync(FULL, out[r]);
    k += __popc(om[r]);
  }
  if (k == 0) return CLIP_NONE;
  if (k == c.nv) return CLIP_EMPTY;
  // a plane slot for h; reclaim slots of planes no kept vertex uses when full
  int h = -1;
#pragma unroll
  for (int w = NPW - 1; w >= 0; w--)
    if (c.freem[w]) h = 32 * w + __ffs(c.freem[w]) - 1;
  if (h < 0) {
    uint32_t lm[NPW];
#pragma unroll
    for (int w = 0; w < NPW; w++) lm[w] = 0;
#pragma unroll
    for (int r = 0; r < VPL; r++)
      if (c.vt[r] != kEmptyTri && !out[r]) {
#pragma unroll
        for (int b = 0; b < 3; b++) {
          uint32_t f = (c.vt[r] >> (8 * b)) & 255u;
#pragma unroll
          for (int w = 0; w < NPW; w++)
            if ((f >> 5) == (uint32_t)w) lm[w] |= 1u << (f & 31u);
        }
      }
#pragma unroll
    for (int w = NPW - 1; w >= 0; w--) {
      c.freem[w] = ~__reduce_or_sync(FULL, lm[w]);
      if (c.freem[w]) h = 32 * w + __ffs(c.freem[w]) - 1;
    }
    if (h < 0) return CLIP_OVERFLOW;
  }
#pragma unroll
  for (int w = 0; w < NPW; w++)
    if ((h >> 5) == w) c.freem[w] &= ~(1u << (h & 31));
  if (lane == 0) {
    S.pl[h] = make_float4(H.nx, H.ny, H.nz, H.b);
    S.pe[h] = H.e;
    S.pid[h] = hpid;
  }
  // step 2: the outside vertices
  int base = 0;
#pragma unroll
  for (int r = 0; r < VPL; r++) {
    if (out[r]) S.otri[base + __popc(om[r] & lt)] = c.vt[r];
    base += __popc(om[r]);
  }
  __syncwarp();
  // step 3: every directed pair (a,b) of an outside vertex whose reverse
  // (b,a) is in no other outside vertex is a hole edge -> vertex (a,b,h)
  int m = 0;
  const int E = 3 * k;
  for (int e0 = 0; e0 < E; e0 += 32) {
    int e = e0 + (int)lane;
    bool isnew = false;
    uint32_t a = 0, b = 0;
    if (e < E) {
      uint32_t T = S.otri[e / 3];
      uint32_t U = T | (T << 24);
      uint32_t ab = (U >> (8 * (e % 3))) & 0xffffu;
      a = ab & 255u;
      b = ab >> 8;
      uint32_t q = b | (a << 8);
      bool interior = false;
      for (int v = 0; v < k; v++) {
        uint32_t T2 = S.otri[v];
        uint32_t U2 = T2 | (T2 << 24);
        if ((U2 & 0xffffu) == q || ((U2 >> 8) & 0xffffu) == q || ((U2 >> 16) & 0xffffu) == q) {
          interior = true;
          break;
        }
      }
      isnew = !interior;
    }
    uint32_t nm = __ballot_sync(FULL, isnew);
    if (isnew) {
      int slot = m + __popc(nm & lt);
      if (slot < VCAP) {
        PlaneT<float> A = load_plane(S, (int)a), B = load_plane(S, (int)b);
        float x, y, z, ev;
        vertex3<float>(A, B, H, x, y, z, ev);
        S.nvp[slot] = make_float4(x, y, z, ev);
        S.nvt[slot] = a | (b << 8) | ((uint32_t)h << 16);
      }
    }
    m += __popc(nm);
  }
  if (counters) ct.newv += m;
  if (c.nv - k + m > VCAP) return CLIP_OVERFLOW;
  __syncwarp();
  // step 4: new vertices take the freed and empty slots
  int fbase = 0;
#pragma unroll
  for (int r = 0; r < VPL; r++) {
    bool fr = (c.vt[r] == kEmptyTri) || out[r];
    uint32_t fm = __ballot_sync(FULL, fr);
    if (fr) {
      int idx = fbase + __popc(fm & lt);
      if (idx < m) {
        float4 t = S.nvp[idx];
        c.vx[r] = t.x;
        c.vy[r] = t.y;
        c.vz[r] = t.z;
        c.ve[r] = t.w;
        c.vt[r] = S.nvt[idx];
      } else {
        c.vt[r] = kEmptyTri;
      }
    }
    fbase += __popc(fm);
  }
  c.nv = c.nv - k + m;
  __syncwarp();
  return CLIP_DONE;
}


// Start a cell as the box: 6 planes, 8 corners (App. B "Initialization").
template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ void init_cell(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP>& S) {
  constexpr int NPW = Cell<VPL, PCAP, QPL>::NPW;
  const unsigned lane = lane_id();
  if (lane < 6) {
    PlaneT<float> B = box_plane<float>((int)lane, c.me.x, c.me.y, c.me.z, c.lo, c.hi);
    S.pl[lane] = make_float4(B.nx, B.ny, B.nz, B.b);
    S.pe[lane] = B.e;
    S.pid[lane] = -1 - (int)lane;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < VPL; r++) c.vt[r] = kEmptyTri;
  if (lane < 8) {
    int sx = lane & 1, sy = (lane >> 1) & 1, sz = (lane >> 2) & 1;
    int a = sx, b = 2 + sy, d = 4 + sz;
    if ((sx + sy + sz) & 1) {
      int t = b;
      b = d;
      d = t;
    }
    PlaneT<float> A = load_plane(S, a), B = load_plane(S, b), D = load_plane(S, d);
    vertex3<float>(A, B, D, c.vx[0], c.vy[0], c.vz[0], c.ve[0]);
    c.vt[0] = (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)d << 16);
  }
  c.nv = 8;
#pragma unroll
  for (int w = 0; w < NPW; w++) c.freem[w] = 0xffffffffu;
  c.freem[0] = ~63u;
#pragma unroll
  for (int r = 0; r < QPL; r++) c.qocc[r] = -1;
  c.seq = 0;
  c.dirty = false;
  recompute_aabb(c);
}

// Compact the vertices into shared memory (S.nvp / S.nvt, in slot order),
// return their count, their coordinate sums and the planes they reference.
template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ int gather_vertices(const Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP>& S, float& sx,
                                               float& sy, float& sz, uint32_t (&alive)[PCAP / 32]) {
  constexpr int NPW = PCAP / 32;
  const unsigned lt = lanemask_lt();
  int vb = 0;
  sx = sy = sz = 0.f;
  uint32_t lm[NPW];
#pragma unroll
  for (int w = 0; w < NPW; w++) lm[w] = 0;
#pragma unroll
  for (int r = 0; r < VPL; r++) {
    bool v = c.vt[r] != kEmptyTri;
    uint32_t m = __ballot_sync(FULL, v);
    if (v) {
      int idx = vb + __popc(m & lt);
      S.nvp[idx] = make_float4(c.vx[r], c.vy[r], c.vz[r], c.ve[r]);
      S.nvt[idx] = c.vt[r];
      sx += c.vx[r];
      sy += c.vy[r];
      sz += c.vz[r];
#pragma unroll
      for (int b = 0; b < 3; b++) {
        uint32_t f = (c.vt[r] >> (8 * b)) & 255u;
#pragma unroll
        for (int w = 0; w < NPW; w++)
          if ((f >> 5) == (uint32_t)w) lm[w] |= 1u << (f & 31u);
      }
    }
    vb += __popc(m);
  }
#pragma unroll
  for (int w = 0; w < NPW; w++) alive[w] = __reduce_or_sync(FULL, lm[w]);
  sx = warp_sumf(sx);
  sy = warp_sumf(sy);
  sz = warp_sumf(sz);
  __syncwarp();
  return vb;
}

// Index of the vertex holding the cyclic plane pair q = (x | y<<8), i.e.
// the other end of the edge x∩y seen from a vertex holding (y, x).
__device__ __forceinline__ bool tri_has_pair(uint32_t T, uint32_t q) {
  uint32_t U = T | (T << 24);
  return (U & 0xffffu) == q || ((U >> 8) & 0xffffu) == q || ((U >> 16) & 0xffffu) == q;
}

}  // namespace vd
