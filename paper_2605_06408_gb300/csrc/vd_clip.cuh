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

// Per-warp event counters, kept in shared memory (not registers); uniform
// events are counted by lane 0, per-lane events with shared atomics.
struct WarpCounters {
  unsigned long long cand, clips, nodes, vtests, newv;
  unsigned fp64, fp64amb, refv, refvol;
};

template <int VPL, int PCAP, int QPL>
struct WarpSmem {
  float4 pl[PCAP];   // n^x, n^y, n^z, b^ (local frame)
  float pe[PCAP];    // offset error bound per plane
  int pid[PCAP];     // sorted site index, or -1-f for box face f
  uint32_t otri[32 * VPL];
  float4 nvp[32 * VPL];
  uint32_t nvt[32 * VPL];
  // best-first queue, dense in [0, qn): lower bound, node reference,
  // occupied-octant bits | push sequence << 8
  float qlb[32 * QPL];
  int qref[32 * QPL];
  int qocc[32 * QPL];
  float rtab[64];          // cell radius per occupied-octant mask
  int knn[kKnn];           // KNN warm start: the cell's nearest sites (sorted indices, -1 = none)
  unsigned amb_mark;       // FP64-ambiguous sign count before the current cell
  int anchor[PCAP];        // FP64 integration: one vertex per face
  double vd64[3 * 32 * VPL];  // FP64 integration: vertex positions
  WarpCounters ct;
};

struct Counters {
  long long cand, clips, nodes, vtests, newv, fp64, fp64amb, refv, refvol;
};

// A new vertex whose FP32 error bound exceeds this fraction of its |x|_1
// (nearly parallel planes) is re-solved in FP64 from the original inputs.
constexpr float kRefineRel = 8192.0f * 5.9604644775390625e-8f;

template <int VPL, int PCAP, int QPL>
struct Cell {
  static constexpr int VCAP = 32 * VPL;
  static constexpr int NPW = PCAP / 32;
  // vertices (per lane)
  float vx[VPL], vy[VPL], vz[VPL], ve[VPL];
  uint32_t vt[VPL];
  // warp-uniform state
  float4 me;
  const float* box;  // the set's box: lo[3] then hi[3] (global memory)
  float alo[3], ahi[3];
  float sc[3], srad;  // bounding sphere of the cell (local frame)
  int nv;
  uint32_t freem[NPW];
  int qn, seq;
  bool dirty;
  bool fp64;  // FP64 re-evaluation of ambiguous predicates, vertices and volumes
};

template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ PlaneT<float> load_plane(const WarpSmem<VPL, PCAP, QPL>& S, int k) {
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

// ---------------------------------------------------------------- FP64 re-evaluation
//
// The FP64 steps take the planes unnormalised, n.x <= b with n = q - p and
// b = (|n|^2 + w_p - w_q) / 2 (x in the frame of the site p; a box face has
// a unit axis normal and b = hi - p or p - lo): the same half-spaces as the
// normalised planes of Eq. 2, formed without a square root or a division.
// The vertex of three planes is then one Cramer solve, x = num / W, and the
// sign of a fourth plane H at that vertex is sign(W) sign(n_H.num - b_H W),
// a polynomial in the inputs with no division at all. Each quantity carries
// an a-priori bound on its rounding error, from the magnitudes below
// (n1 = |n|_1, bm = |n|^2 + |w_p| + |w_q| bounds |b| and its error /4u):
// every entry of n is off by at most u|n_i|, b by at most 4u bm.
struct Plane64u {
  double nx, ny, nz, b, n1, bm;
};

__device__ __forceinline__ Plane64u plane64u(int id, const float4& me, const float* lo, const float* hi,
                                             const float4* __restrict__ sites) {
  Plane64u P;
  if (id >= 0) {
    const float4 q = sites[id];
    P.nx = (double)q.x - (double)me.x;
    P.ny = (double)q.y - (double)me.y;
    P.nz = (double)q.z - (double)me.z;
    const double nn = fma(P.nx, P.nx, fma(P.ny, P.ny, P.nz * P.nz));
    P.b = 0.5 * (nn + ((double)me.w - (double)q.w));
    P.n1 = fabs(P.nx) + fabs(P.ny) + fabs(P.nz);
    P.bm = nn + fabs((double)me.w) + fabs((double)q.w);
  } else {
    const int f = -1 - id, ax = f >> 1;
    const double s = (f & 1) ? -1.0 : 1.0;
    const double pc = ax == 0 ? (double)me.x : (ax == 1 ? (double)me.y : (double)me.z);
    P.nx = ax == 0 ? s : 0.0;
    P.ny = ax == 1 ? s : 0.0;
    P.nz = ax == 2 ? s : 0.0;
    const double bound = (f & 1) ? (double)lo[ax] : (double)hi[ax];
    P.b = (f & 1) ? (pc - bound) : (bound - pc);
    P.n1 = 1.0;
    P.bm = fabs(pc) + fabs(bound);
  }
  return P;
}

// Cramer parts of the vertex of (A, B, C): num = b_A (n_B x n_C) + b_B (n_C x n_A)
// + b_C (n_A x n_B), W = n_A.(n_B x n_C), with bounds dW on |W - W_exact| and
// dnum on each |num_i - num_i,exact| (cross-product entries off by at most
// 4u n1 n1 with the input errors, sums by 3u of their terms; the constants
// are doubled).
struct Cramer64 {
  double nx, ny, nz, W, dW, dnum, mnum;
};

__device__ __forceinline__ Cramer64 cramer64(const Plane64u& A, const Plane64u& B, const Plane64u& C) {
  const double u = Num<double>::u;
  const double c1x = fma(B.ny, C.nz, -B.nz * C.ny), c1y = fma(B.nz, C.nx, -B.nx * C.nz),
               c1z = fma(B.nx, C.ny, -B.ny * C.nx);
  const double c2x = fma(C.ny, A.nz, -C.nz * A.ny), c2y = fma(C.nz, A.nx, -C.nx * A.nz),
               c2z = fma(C.nx, A.ny, -C.ny * A.nx);
  const double c3x = fma(A.ny, B.nz, -A.nz * B.ny), c3y = fma(A.nz, B.nx, -A.nx * B.nz),
               c3z = fma(A.nx, B.ny, -A.ny * B.nx);
  Cramer64 R;
  R.W = fma(A.nx, c1x, fma(A.ny, c1y, A.nz * c1z));
  R.nx = fma(A.b, c1x, fma(B.b, c2x, C.b * c3x));
  R.ny = fma(A.b, c1y, fma(B.b, c2y, C.b * c3y));
  R.nz = fma(A.b, c1z, fma(B.b, c2z, C.b * c3z));
  const double bc = B.n1 * C.n1, ca = C.n1 * A.n1, ab = A.n1 * B.n1;
  R.mnum = fabs(A.b) * bc + fabs(B.b) * ca + fabs(C.b) * ab;  // bounds every |num_i| term sum
  R.dW = 16.0 * u * (A.n1 * bc);
  R.dnum = 16.0 * u * R.mnum + 8.0 * u * (A.bm * bc + B.bm * ca + C.bm * ab);
  return R;
}

// Vertex of (A, B, C) and a bound E on |x - x_exact|_1 (first order, with
// |W| kept above 64 dW so that the second-order terms stay below a third of
// it; E = inf otherwise).
__device__ __forceinline__ void vertex64u(const Plane64u& A, const Plane64u& B, const Plane64u& C, double& x,
                                          double& y, double& z, double& E) {
  const double u = Num<double>::u;
  const Cramer64 R = cramer64(A, B, C);
  const double iw = 1.0 / R.W;
  x = R.nx * iw;
  y = R.ny * iw;
  z = R.nz * iw;
  const double x1 = fabs(x) + fabs(y) + fabs(z);
  if (!(fabs(R.W) > 64.0 * R.dW) || !(x1 < 1e300)) {
    E = INFINITY;
  } else {
    E = 1.5 * (3.0 * R.dnum + x1 * R.dW) / fabs(R.W) + 4.0 * u * x1;
  }
}

// Does the vertex of (A, B, C) lie strictly outside H? D = n_H.num - b_H W has
// the sign of (n_H.x - b_H) W; its error is at most dD (the errors of num and
// W carried through, n_H and b_H off by u n1 and 4u bm, and the rounding of
// the sums); amb is set when |D| <= dD or W's own sign is not certain, and
// the FP64 sign is taken then.
__device__ __forceinline__ bool side64u(const Plane64u& A, const Plane64u& B, const Plane64u& C, const Plane64u& H,
                                        bool& amb) {
  const double u = Num<double>::u;
  const Cramer64 R = cramer64(A, B, C);
  const double D = fma(H.nx, R.nx, fma(H.ny, R.ny, fma(H.nz, R.nz, -H.b * R.W)));
  const double mW = A.n1 * B.n1 * C.n1;
  const double dD = 2.0 * (H.n1 * (R.dnum + 4.0 * u * R.mnum) + fabs(H.b) * R.dW + 8.0 * u * H.bm * mW +
                           4.0 * u * (H.n1 * R.mnum + fabs(H.b) * mW));
  amb = !(fabs(R.W) > R.dW) || !(fabs(D) > dD);
  return R.W > 0.0 ? D > 0.0 : D < 0.0;
}

// FP64 re-evaluation of "vertex tri lies outside the plane of site hpid".
template <int VPL, int PCAP, int QPL>
static __device__ __noinline__ bool resolve64(WarpSmem<VPL, PCAP, QPL>& S, uint32_t tri, int hpid, float4 me,
                                              const float* lo, const float* hi, const float4* __restrict__ sites) {
  const Plane64u A = plane64u(S.pid[tri & 255u], me, lo, hi, sites);
  const Plane64u B = plane64u(S.pid[(tri >> 8) & 255u], me, lo, hi, sites);
  const Plane64u C = plane64u(S.pid[(tri >> 16) & 255u], me, lo, hi, sites);
  const Plane64u H = plane64u(hpid, me, lo, hi, sites);
  bool amb = false;
  const bool out = side64u(A, B, C, H, amb);
  if (amb) atomicAdd(&S.ct.fp64amb, 1u);
  return out;
}

// FP64 re-solve of the vertex of planes (pa, pb, ph) (plane ids: sorted
// site index or -1-face); the FP32 result's bound becomes the FP64 bound plus
// one rounding to float and the terms of a later FP32 sign test.
static __device__ __noinline__ void refine_vertex(int pa, int pb, int ph, float4 me, const float* lo, const float* hi,
                                           const float4* __restrict__ sites, float& x, float& y, float& z,
                                           float& e) {
  const Plane64u A = plane64u(pa, me, lo, hi, sites), B = plane64u(pb, me, lo, hi, sites),
                 H = plane64u(ph, me, lo, hi, sites);
  double X, Y, Z, E;
  vertex64u(A, B, H, X, Y, Z, E);
  x = (float)X;
  y = (float)Y;
  z = (float)Z;
  float x1 = fabsf(x) + fabsf(y) + fabsf(z);
  e = (E < 1e30) ? (float)(E * (1.0 + 1e-6)) + 12.0f * Num<float>::u * x1 * 1.0001f : INFINITY;
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

// Upper bound on the cell's extent toward any site in the octants `occ`:
// the directional AABB radius, capped by the bounding sphere's reach
// |center| + radius (valid in every direction).
__device__ __forceinline__ float cell_radius(int occ, const float* alo, const float* ahi, const float* sc, float srad,
                                             int cull_mode) {
  float R = sqrtf(dir_radius2(occ, alo, ahi, cull_mode));
  if (cull_mode == 0) R = fminf(R, sqrtf(sc[0] * sc[0] + sc[1] * sc[1] + sc[2] * sc[2]) + srad);
  return R;
}

// Cell radius for each of the 64 occupied-octant masks (see cell_radius),
// refreshed whenever the cell's bounds change so that node tests and queue
// re-tests are one table lookup.
__device__ __forceinline__ void fill_rtab(float* rtab, const float* alo, const float* ahi, const float* sc, float srad,
                                          int cull_mode) {
  for (int o = (int)lane_id(); o < 64; o += 32) rtab[o] = cell_radius(o, alo, ahi, sc, srad, cull_mode);
  __syncwarp();
}

template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ void recompute_aabb(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, int cull_mode) {
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
    c.sc[k] = 0.5f * (c.alo[k] + c.ahi[k]);
  }
  float r2 = 0.0f;
#pragma unroll
  for (int r = 0; r < VPL; r++)
    if (c.vt[r] != kEmptyTri) {
      float dx = c.vx[r] - c.sc[0], dy = c.vy[r] - c.sc[1], dz = c.vz[r] - c.sc[2];
      r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
  c.srad = (sqrtf(warp_maxf(r2)) + em) * (1.0f + kCullPad);
  fill_rtab(S.rtab, c.alo, c.ahi, c.sc, c.srad, cull_mode);
}

// Test of one BVH child box [lo.xyz, hi.xyz] with maximum weight lo.w
// (Sec. 4.2.2). For a site j in the box at distance D in [dmin, dmax],
// d_ij = D/2 + (w_i - w_j)/(2D) >= f(D) = D/2 + c/(2D), c = w_i - w_max.
// f is increasing for c <= 0, so LB = f(dmin) -- the paper's bound; for
// c > 0 it is convex with its minimum at sqrt(c), so LB = f(clamp(sqrt c,
// dmin, dmax)) (tighter than the paper's dmin/2 for heavy sites). Culled
// iff LB exceeds the cell radius over the octants the box occupies.
// Returns keep; lb is a safe (padded) LB, key the best-first key LB - R.
// Radius lookup rad(occ) gives the cell radius over the occupied octants.
template <typename RadiusOf>
__device__ __forceinline__ bool node_test_r(float4 lo, float4 hi, float4 me, RadiusOf rad, int cull_mode, float& lb,
                                            int& occ, float& key) {
  float rl[3] = {lo.x - me.x, lo.y - me.y, lo.z - me.z};
  float rh[3] = {hi.x - me.x, hi.y - me.y, hi.z - me.z};
  float d2 = 0.0f, f2 = 0.0f;
  occ = 0;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float dk = fmaxf(fmaxf(rl[k], -rh[k]), 0.0f);
    float fk = fmaxf(fabsf(rl[k]), fabsf(rh[k]));
    d2 = fmaf(dk, dk, d2);
    f2 = fmaf(fk, fk, f2);
    occ |= (rh[k] >= 0.0f ? 1 : 0) << (2 * k);
    occ |= (rl[k] <= 0.0f ? 1 : 0) << (2 * k + 1);
  }
  float R = rad(occ);
  float c = me.w - lo.w;
  float D = sqrtf(d2);
  if (c > 0.0f) D = fminf(fmaxf(sqrtf(c), D), sqrtf(f2) * (1.0f + kCullPad));
  if (!(D > 0.0f)) {
    lb = -INFINITY;
    key = -R;
    return true;
  }
  float D2 = D * D;
  // one approximate reciprocal for both quotients: its error (a few ulp)
  // is far inside the relative pad of 1e-5 that keeps lb a lower bound
  const float inv = __fdividef(0.5f, D);
  lb = (D2 + c - kCullPad * (D2 + fabsf(me.w) + fabsf(lo.w))) * inv;
  key = (D2 + c) * inv - R;
  if (cull_mode == 2) return true;
  return !(lb > R * (1.0f + kCullPad));
}

__device__ __forceinline__ bool node_test(float4 lo, float4 hi, float4 me, const float* rtab, int cull_mode,
                                          float& lb, int& occ, float& key) {
  return node_test_r(lo, hi, me, [&](int o) { return rtab[o]; }, cull_mode, lb, occ, key);
}

// Cone bound of a child box [lo, hi] (local frame after subtracting the
// site): every site j in the box has its plane normal n_j within the cone of
// axis u (toward the box centre) and half-angle theta (the cone tangent to
// the box's circumscribed ball), and its plane can cut the cell only if
// d_ij < h(n_j), the cell's support in direction n_j. The support function
// is Lipschitz with constant max|v|, so h(n_j) <= h(u) + 2 sin(theta/2) max|v|.
// Returns false when the cone is every direction (the site inside the ball).
struct Cone {
  float ux, uy, uz, slack_per_r;  // axis, 2 sin(theta/2)
};
__device__ __forceinline__ bool node_cone(float4 lo, float4 hi, float4 me, Cone& k) {
  const float cx = 0.5f * (lo.x + hi.x) - me.x, cy = 0.5f * (lo.y + hi.y) - me.y, cz = 0.5f * (lo.z + hi.z) - me.z;
  const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
  const float d2 = cx * cx + cy * cy + cz * cz;
  const float r2 = (hx * hx + hy * hy + hz * hz) * (1.0f + 1e-4f);
  if (!(d2 > 1.0001f * r2) || !(d2 > 0.0f)) return false;
  const float id = rsqrtf(d2);
  k.ux = cx * id;
  k.uy = cy * id;
  k.uz = cz * id;
  // cos(theta) = sqrt(1 - r^2/d^2); 2 sin(theta/2) = sqrt(2 - 2 cos(theta))
  const float ct = sqrtf(fmaxf(0.0f, 1.0f - r2 / d2));
  k.slack_per_r = sqrtf(fmaxf(0.0f, 2.0f - 2.0f * ct)) * (1.0f + 1e-4f) + 1e-6f;
  return true;
}
// Culled iff the padded LB exceeds the cone bound (support h in direction
// u, plus the vertex error bound and the Lipschitz slack).
__device__ __forceinline__ bool cone_culls(float lb, float h, float em, float rmax, const Cone& k) {
  const float R = h + em + k.slack_per_r * rmax;
  return lb > R * (1.0f + kCullPad) + kCullPad * rmax;
}

template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ bool queue_push(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, float lb, int ref,
                                           int occ) {
  if (c.qn >= 32 * QPL) return false;
  if (lane_id() == 0) {
    S.qlb[c.qn] = lb;
    S.qref[c.qn] = ref;
    S.qocc[c.qn] = occ | (c.seq << 8);
  }
  c.qn++;
  c.seq++;
  __syncwarp();
  return true;
}

// Pop the most promising entry still valid under the current cell bounds
// (Alg. 1 backtracking: re-test with the shrunken radii; entries that now
// fail are dropped). The queue is kept unsorted and the popped slot takes
// the last entry (App. A.5); the minimum is one redux.sync over the lanes.
// Depth-first mode pops the newest entry.
template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ bool queue_pop(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, int cull_mode,
                                          int traversal, int& ref) {
  const unsigned lane = lane_id(), lt = lanemask_lt();
  int live = 0;
  uint32_t bestk = 0xffffffffu;
  int besti = 0x7fffffff;
  for (int base = 0; base < c.qn; base += 32) {
    int i = base + (int)lane;
    bool ok = false;
    float lb = 0.f;
    int rf = 0, oc = 0;
    uint32_t key = 0xffffffffu;
    if (i < c.qn) {
      lb = S.qlb[i];
      rf = S.qref[i];
      oc = S.qocc[i];
      float R = S.rtab[oc & 63];
      ok = cull_mode == 2 || !(lb > R * (1.0f + kCullPad));
      key = traversal == 0 ? f2o(lb - R) : (0xfffffffeu - (uint32_t)(oc >> 8));
    }
    uint32_t km = __ballot_sync(FULL, ok);
    int dst = live + __popc(km & lt);
    __syncwarp();
    if (ok) {
      S.qlb[dst] = lb;
      S.qref[dst] = rf;
      S.qocc[dst] = oc;
      if (key < bestk) {
        bestk = key;
        besti = dst;
      }
    }
    live += __popc(km);
    __syncwarp();
  }
  c.qn = live;
  uint32_t mn = __reduce_min_sync(FULL, bestk);
  if (live == 0 || mn == 0xffffffffu) return false;
  int idx = (int)__reduce_min_sync(FULL, bestk == mn ? (uint32_t)besti : 0x7fffffffu);
  ref = S.qref[idx];
  __syncwarp();
  if (lane == 0) {
    int last = c.qn - 1;
    S.qlb[idx] = S.qlb[last];
    S.qref[idx] = S.qref[last];
    S.qocc[idx] = S.qocc[last];
  }
  c.qn--;
  __syncwarp();
  return true;
}

enum { CLIP_NONE = 0, CLIP_DONE = 1, CLIP_EMPTY = 2, CLIP_OVERFLOW = 3, CLIP_OVF_PLANES = 4 };
enum { OVF_QUEUE = 0, OVF_VERTICES = 1, OVF_PLANES = 2, OVF_NEIGHBORS = 3 };

// Clip the cell by plane H of site hpid (App. B "Clipping by a half-space").
template <int VPL, int PCAP, int QPL>
__device__ int clip_cell(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, const PlaneT<float>& H, int hpid,
                         const float4* __restrict__ sites, bool counters) {
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
      if (c.fp64 && ambiguous<float>(s, c.ve[r], H.e)) {
        atomicAdd(&S.ct.fp64, 1u);
        out[r] = resolve64(S, c.vt[r], hpid, c.me, c.box, c.box + 3, sites);
      }
    }
  }
  if (counters && lane == 0) S.ct.vtests += c.nv;
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
    if (h < 0) return CLIP_OVF_PLANES;
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
        if (c.fp64 && !(ev <= kRefineRel * (fabsf(x) + fabsf(y) + fabsf(z)))) {
          refine_vertex(S.pid[a], S.pid[b], hpid, c.me, c.box, c.box + 3, sites, x, y, z, ev);
          atomicAdd(&S.ct.refv, 1u);
        }
        S.nvp[slot] = make_float4(x, y, z, ev);
        S.nvt[slot] = a | (b << 8) | ((uint32_t)h << 16);
      }
    }
    m += __popc(nm);
  }
  if (counters && lane == 0) S.ct.newv += m;
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


// Candidate pre-test of Sec. 4.2.1: the plane n.x <= beta can cut the cell
// only if it cuts the cell's AABB, i.e. n.c_o > beta for the AABB corner c_o
// of n's octant (the exact support of the box in direction n; the paper's
// per-octant corner distance |c_o| bounds it from above).
__device__ __forceinline__ bool candidate_test(float nx, float ny, float nz, float nn, float beta, float wi,
                                               float wj, const float* alo, const float* ahi, const float* sc,
                                               float srad, int cull_mode) {
  if (cull_mode == 2) return true;
  float n[3] = {nx, ny, nz};
  float pad = 0.5f * (nn + fabsf(wi) + fabsf(wj));
  if (cull_mode == 1) {
    float R = sqrtf(dir_radius2(0, alo, ahi, 1));
    float len = sqrtf(nn);
    pad = kCullPad * (pad + len * R);
    return len * R * (1.0f + kCullPad) > beta - pad;
  }
  float sup = 0.0f, mag = 0.0f, n1 = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float t = n[k] > 0.0f ? n[k] * ahi[k] : (n[k] < 0.0f ? n[k] * alo[k] : 0.0f);
    sup += t;
    mag += fabsf(t);
    n1 += fabsf(n[k]);
  }
  if (!(sup > beta - kCullPad * (pad + mag))) return false;
  // bounding sphere: n.sc + srad |n| > beta  <=>  srad^2 nn > (beta - n.sc)^2 when beta > n.sc
  float ns = n[0] * sc[0] + n[1] * sc[1] + n[2] * sc[2];
  float rhs = beta - ns - kCullPad * (pad + n1 * (fabsf(sc[0]) + fabsf(sc[1]) + fabsf(sc[2]) + srad));
  return rhs <= 0.0f || srad * srad * nn > rhs * rhs;
}

// Start a cell as the box: 6 planes, 8 corners (App. B "Initialization").
template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ void init_cell(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, int cull_mode) {
  constexpr int NPW = Cell<VPL, PCAP, QPL>::NPW;
  const unsigned lane = lane_id();
  if (lane < 6) {
    PlaneT<float> B = box_plane<float>((int)lane, c.me.x, c.me.y, c.me.z, c.box, c.box + 3);
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
    // box corner: the three axis-aligned planes meet at (+-b) exactly (the
    // solve of vertex3 has determinant 1 and unit cofactors here), and its
    // error bound reduces to the terms below (vertex3's bound with W = 1)
    const float4 Px = S.pl[sx], Py = S.pl[2 + sy], Pz = S.pl[4 + sz];
    const float u = Num<float>::u;
    c.vx[0] = sx ? -Px.w : Px.w;
    c.vy[0] = sy ? -Py.w : Py.w;
    c.vz[0] = sz ? -Pz.w : Pz.w;
    const float x1 = fabsf(c.vx[0]) + fabsf(c.vy[0]) + fabsf(c.vz[0]);
    const float sumE = S.pe[sx] + S.pe[2 + sy] + S.pe[4 + sz];
    const float ep = (1.75f * sumE + (5.25f * 8.0f * u + 9.0f * u) * x1 + 6.0f * u * x1) + u * x1;
    c.ve[0] = x1 < 1e30f ? 1.1f * ep + (8.0f * u + 3.0f * u) * x1 : INFINITY;
    c.vt[0] = (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)d << 16);
  }
  c.nv = 8;
#pragma unroll
  for (int w = 0; w < NPW; w++) c.freem[w] = 0xffffffffu;
  c.freem[0] = ~63u;
  c.qn = 0;
  c.seq = 0;
  c.dirty = false;
  recompute_aabb(c, S, cull_mode);
}

// Compact the vertices into shared memory (S.nvp / S.nvt, in slot order),
// return their count, their coordinate sums and the planes they reference.
template <int VPL, int PCAP, int QPL>
__device__ __forceinline__ int gather_vertices(const Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, float& sx,
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

// A cell's FP32 volume is accepted unless an estimate of its error says
// otherwise: with L the largest vertex distance from the site and S the
// summed |area| of the integration triangles, the volume error scales like
// u L S; cells with L S > 36 V (a site far from its own cell, or a sliver)
// or with a vertex bound above 4096 u L are integrated again in FP64.
__device__ __forceinline__ bool volume_needs_fp64(float V, float L, float Sabs, float emax) {
  return !(V > 0.f) || (L * Sabs > 36.f * V) || (emax > 4096.f * Num<float>::u * L);
}

__device__ __forceinline__ void vertex64(uint32_t a, uint32_t b, uint32_t c, const int* pid, float4 me, const float* lo,
                                         const float* hi, const float4* __restrict__ sites, double& x, double& y,
                                         double& z) {
  double e;
  vertex64u(plane64u(pid[a], me, lo, hi, sites), plane64u(pid[b], me, lo, hi, sites),
            plane64u(pid[c], me, lo, hi, sites), x, y, z, e);
}

// Volume and first moment about c of the register-path polytope gathered in
// S.nvt (slot order, nv vertices), in FP64: every vertex is re-solved once
// from the original inputs (kept in S.vd64), and each face's fan is anchored
// at one of its own vertices (its lowest index), so the integration uses no
// point that is not a vertex of the cell.
template <int VPL, int PCAP, int QPL>
__device__ __noinline__ void volume_fp64(WarpSmem<VPL, PCAP, QPL>& S, int nv, float4 me, const float* lo,
                                         const float* hi, const float4* __restrict__ sites, double cx, double cy,
                                         double cz, double& V, double& Mx, double& My, double& Mz) {
  const unsigned lane = lane_id();
  for (int f = (int)lane; f < PCAP; f += 32) S.anchor[f] = 0x7fffffff;
  __syncwarp();
  for (int t = (int)lane; t < nv; t += 32) {
    uint32_t T = S.nvt[t];
    double x, y, z;
    vertex64(T & 255u, (T >> 8) & 255u, (T >> 16) & 255u, S.pid, me, lo, hi, sites, x, y, z);
    S.vd64[3 * t] = x - cx;
    S.vd64[3 * t + 1] = y - cy;
    S.vd64[3 * t + 2] = z - cz;
    atomicMin(&S.anchor[T & 255u], t);
    atomicMin(&S.anchor[(T >> 8) & 255u], t);
    atomicMin(&S.anchor[(T >> 16) & 255u], t);
  }
  __syncwarp();
  V = Mx = My = Mz = 0.0;
  for (int it = (int)lane; it < 3 * nv; it += 32) {
    int t = it / 3, rho = it % 3;
    uint32_t T = S.nvt[t];
    uint32_t U = T | (T << 24);
    uint32_t xy = (U >> (8 * rho)) & 0xffffu;
    uint32_t fx = xy & 255u, fy = xy >> 8;
    uint32_t q = fy | (fx << 8);
    int u = 0;
    while (u < nv && !tri_has_pair(S.nvt[u], q)) u++;
    int g = S.anchor[fy];
    if (u >= nv || g == t || g == u) continue;  // triangles through the anchor vanish
    const double* A = &S.vd64[3 * g];
    const double* B = &S.vd64[3 * t];
    const double* C = &S.vd64[3 * u];
    double det = A[0] * (B[1] * C[2] - B[2] * C[1]) + A[1] * (B[2] * C[0] - B[0] * C[2]) +
                 A[2] * (B[0] * C[1] - B[1] * C[0]);
    V += det;
    Mx += det * (A[0] + B[0] + C[0]);
    My += det * (A[1] + B[1] + C[1]);
    Mz += det * (A[2] + B[2] + C[2]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    V += __shfl_xor_sync(FULL, V, o);
    Mx += __shfl_xor_sync(FULL, Mx, o);
    My += __shfl_xor_sync(FULL, My, o);
    Mz += __shfl_xor_sync(FULL, Mz, o);
  }
  V /= 6.0;
  Mx /= 24.0;
  My /= 24.0;
  Mz /= 24.0;
  __syncwarp();
}

}  // namespace vd
