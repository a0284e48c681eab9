// vd_backward.cu -- adjoint of the forward build (no counterpart in the
// paper, which constructs the diagram only).
//
// L = sum_i gv_i V_i + gc_i . g_i (V = volume, g = centroid). With the cell
// combinatorics held fixed, only site-site faces move: on face F_ij of cell
// i (distance D = |p_j - p_i|, n = p_j - p_i, local coordinates x~ = x - p_i)
// the boundary's normal speed is (n - x~).dp_j / D, x~.dp_i / D, dw_i / 2D
// and -dw_j / 2D (differentiate |x-p_i|^2 - w_i - |x-p_j|^2 + w_j = 0 and
// divide by its gradient 2D). Reynolds transport then gives, with
// A = area, Am = int x~ dA, S = int x~ x~^T dA over F_ij,
//   dL_i = a' dV + b . dM~,   b = gc_i / V_i,   a' = gv_i - b . g~_i,
//   dV/dp_j = (A n - Am)/D, dV/dp_i = Am/D, dV/dw_i = -dV/dw_j = A/2D,
//   dM~/dp_j = (Am n^T - S)/D, dM~/dp_i = S/D, dM~/dw_i = -dM~/dw_j = Am/2D,
// where M~ = int x~ dV and g~ = M~/V. Each cell is re-clipped from its
// stored neighbour list (no traversal), its faces integrated by the same
// fan tetrahedra as the forward pass, and the face terms scatter-added.
#include "vd_big.cuh"

namespace vd {

template <int VPL, int PCAP>
struct BackSmem {
  WarpSmem<VPL, PCAP, 1> w;
  float acc[PCAP][10];  // per face: A, int y (3), int y y^T (6), y = x~ - c
};

// Scatter one site face's contribution (accumulators A = area, int y,
// int y y^T about the vertex mean c) of cell i to the neighbour j, and add
// the cell's own share to gpi / gwi.
__device__ __forceinline__ void face_gradient(const float* A, float cx, float cy, float cz, float4 me, float4 qj,
                                              int oj, float ap, float b0, float b1, float b2, float* gp, float* gw,
                                              float& gpi0, float& gpi1, float& gpi2, float& gwi) {
  float Ar = A[0];
  float iy[3] = {A[1], A[2], A[3]};
  float Syy[3][3] = {{A[4], A[7], A[8]}, {A[7], A[5], A[9]}, {A[8], A[9], A[6]}};
  float cc[3] = {cx, cy, cz};
  // shift the moments from the vertex mean c to the site p_i
  float Am[3], St[3][3];
#pragma unroll
  for (int p = 0; p < 3; p++) Am[p] = Ar * cc[p] + iy[p];
#pragma unroll
  for (int p = 0; p < 3; p++)
#pragma unroll
    for (int r = 0; r < 3; r++) St[p][r] = Ar * cc[p] * cc[r] + cc[p] * iy[r] + iy[p] * cc[r] + Syy[p][r];
  float n[3] = {qj.x - me.x, qj.y - me.y, qj.z - me.z};
  float D = sqrtf(fmaf(n[0], n[0], fmaf(n[1], n[1], n[2] * n[2])));
  float iD = 1.0f / D;
  float amb = Am[0] * b0 + Am[1] * b1 + Am[2] * b2;
  float Sb[3];
#pragma unroll
  for (int p = 0; p < 3; p++) Sb[p] = St[p][0] * b0 + St[p][1] * b1 + St[p][2] * b2;
#pragma unroll
  for (int p = 0; p < 3; p++) {
    float gj = (ap * (Ar * n[p] - Am[p]) + n[p] * amb - Sb[p]) * iD;
    atomicAdd(&gp[3 * (size_t)oj + p], gj);
  }
  gpi0 += (ap * Am[0] + Sb[0]) * iD;
  gpi1 += (ap * Am[1] + Sb[1]) * iD;
  gpi2 += (ap * Am[2] + Sb[2]) * iD;
  float gwc = (ap * Ar + amb) * 0.5f * iD;
  gwi += gwc;
  if (gw) atomicAdd(&gw[oj], -gwc);
}

// Triangle (g, a, b) of face f (unit normal nf), coordinates relative to
// the vertex mean: add its area, first and second moments to A[0..9].
__device__ __forceinline__ void face_accumulate(float* A, const float* g, const float* a, const float* b, float4 nf) {
  float e1[3] = {a[0] - g[0], a[1] - g[1], a[2] - g[2]};
  float e2[3] = {b[0] - g[0], b[1] - g[1], b[2] - g[2]};
  float cr0 = e1[1] * e2[2] - e1[2] * e2[1], cr1 = e1[2] * e2[0] - e1[0] * e2[2], cr2 = e1[0] * e2[1] - e1[1] * e2[0];
  float al = 0.5f * (cr0 * nf.x + cr1 * nf.y + cr2 * nf.z);
  float s[3] = {g[0] + a[0] + b[0], g[1] + a[1] + b[1], g[2] + a[2] + b[2]};
  atomicAdd(&A[0], al);
#pragma unroll
  for (int k = 0; k < 3; k++) atomicAdd(&A[1 + k], al * s[k] * (1.0f / 3.0f));
  const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int k = 0; k < 6; k++) {
    int p = ii[k], r = jj[k];
    float m2 = g[p] * g[r] + a[p] * a[r] + b[p] * b[r] + s[p] * s[r];
    atomicAdd(&A[4 + k], al * m2 * (1.0f / 12.0f));
  }
}

// Row of the plane through a vertex in the linear system A x = r that
// defines it (world coordinates): a site plane j of cell i is
// 2 (p_j - p_i) . x = |p_j|^2 - |p_i|^2 + w_i - w_j; box face f is
// +-x_axis = bound. nj = p_j - p_i (site) or unused (box).
__device__ __forceinline__ void plane_row(int id, float nx, float ny, float nz, float r[3]) {
  if (id >= 0) {
    r[0] = 2.0f * nx;
    r[1] = 2.0f * ny;
    r[2] = 2.0f * nz;
  } else {
    const int f = -1 - id, ax = f >> 1;
    const float sg = (f & 1) ? -1.0f : 1.0f;
    r[0] = ax == 0 ? sg : 0.0f;
    r[1] = ax == 1 ? sg : 0.0f;
    r[2] = ax == 2 ? sg : 0.0f;
  }
}

// Adjoint of one vertex x (local position v = x - p_i) of cell i defined by
// the planes of ids[0..2]: with lambda = A^-T g (g = dL/dx), implicit
// differentiation of A x = r gives dL/dp_j = 2 lambda_j (p_j - x),
// dL/dw_j = -lambda_j for each site plane j, and dL/dp_i += 2 lambda_j
// (x - p_i), dL/dw_i += lambda_j; box faces do not move.
__device__ __forceinline__ void vertex_gradient(const float4* __restrict__ sites, const int* __restrict__ perm,
                                                float4 me, float4 v, const int ids[3], float g0, float g1, float g2,
                                                float* gp, float* gw, float& gpi0, float& gpi1, float& gpi2,
                                                float& gwi) {
  float n[3][3], r[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    n[k][0] = n[k][1] = n[k][2] = 0.0f;
    if (ids[k] >= 0) {
      const float4 q = sites[ids[k]];
      n[k][0] = q.x - me.x;
      n[k][1] = q.y - me.y;
      n[k][2] = q.z - me.z;
    }
    plane_row(ids[k], n[k][0], n[k][1], n[k][2], r[k]);
  }
  float cr[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float* a = r[(k + 1) % 3];
    const float* b = r[(k + 2) % 3];
    cr[k][0] = a[1] * b[2] - a[2] * b[1];
    cr[k][1] = a[2] * b[0] - a[0] * b[2];
    cr[k][2] = a[0] * b[1] - a[1] * b[0];
  }
  const float det = r[0][0] * cr[0][0] + r[0][1] * cr[0][1] + r[0][2] * cr[0][2];
  if (!(fabsf(det) > 0.0f)) return;
  const float idet = 1.0f / det;
  const float vv[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int k = 0; k < 3; k++) {
    if (ids[k] < 0) continue;
    const float lam = (cr[k][0] * g0 + cr[k][1] * g1 + cr[k][2] * g2) * idet;
    const int oj = perm[ids[k]];
#pragma unroll
    for (int p = 0; p < 3; p++) atomicAdd(&gp[3 * (size_t)oj + p], 2.0f * lam * (n[k][p] - vv[p]));
    if (gw) atomicAdd(&gw[oj], -lam);
    gpi0 += 2.0f * lam * vv[0];
    gpi1 += 2.0f * lam * vv[1];
    gpi2 += 2.0f * lam * vv[2];
    gwi += lam;
  }
}

template <int VPL, int PCAP, int QPL>
__device__ bool back_cell(const BackBuffers& B, BackSmem<VPL, PCAP>& SM, int si) {
  using C = Cell<VPL, PCAP, QPL>;
  constexpr int NPW = C::NPW;
  const CellBuffers& P = B.c;
  WarpSmem<VPL, PCAP, 1>& S = SM.w;
  const unsigned lane = lane_id();
  C c;
  c.me = P.sites[si];
  c.fp64 = P.cfg.precision == 0;
  const int orig_i = P.perm[si];
  const int set = P.nsets > 1 ? (int)(P.keys[si] >> P.set_shift) : 0;
  const SetInfo& SI = P.sets[set];
  c.box = SI.lo;
  const int cnt = P.counts[orig_i];
  if (cnt <= 0) return true;  // empty cell (or no site faces): no moving face
  float sx, sy, sz;
  uint32_t alive[NPW];
  int nv = -1;
  if (B.tape) {
    // the forward's cell from the tape: vertices and face planes (the planes
    // recomputed from their ids exactly as the forward computed them)
    const char* rec = B.tape + (size_t)si * kTapeStride;
    const int4 h = *reinterpret_cast<const int4*>(rec);
    if (h.x == -2) return false;  // a large cell with a record on the large-cell tape
    if (h.x > 0) {
      nv = h.x;
      const int nf = h.y;
      const float4* tv = reinterpret_cast<const float4*>(rec + kTapeVOff);
      const int* tf = reinterpret_cast<const int*>(rec + kTapeFOff);
      sx = sy = sz = 0.f;
      for (int t = (int)lane; t < nv; t += 32) {
        const float4 r = tv[t];
        S.nvp[t] = make_float4(r.x, r.y, r.z, 0.f);
        S.nvt[t] = __float_as_uint(r.w);
        sx += r.x;
        sy += r.y;
        sz += r.z;
      }
      for (int k = (int)lane; k < nf; k += 32) {
        const int id = tf[k];
        PlaneT<float> H;
        if (id >= 0) {
          const float4 q = P.sites[id];
          H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
        } else {
          H = box_plane<float>(-1 - id, c.me.x, c.me.y, c.me.z, c.box, c.box + 3);
        }
        S.pl[k] = make_float4(H.nx, H.ny, H.nz, H.b);
        S.pid[k] = id;
      }
#pragma unroll
      for (int w = 0; w < NPW; w++) alive[w] = nf >= 32 * (w + 1) ? FULL : (nf > 32 * w ? ((1u << (nf - 32 * w)) - 1u) : 0u);
      sx = warp_sumf(sx);
      sy = warp_sumf(sy);
      sz = warp_sumf(sz);
      __syncwarp();
    }
  }
  if (nv < 0) {
  init_cell(c, S, 0);
  const int slot = P.ovf_slot[orig_i];
  if (slot >= 0) return false;  // a long neighbour list: the large-cell adjoint
  const int* row = P.scratch + (size_t)orig_i * P.stride;
  for (int c0 = 0; c0 < cnt; c0 += 32) {
    int t = c0 + (int)lane;
    bool keep = t < cnt;
    int j = 0;
    PlaneT<float> H;
    H.nx = H.ny = H.nz = H.b = H.e = 0.f;
    float dkey = INFINITY;
    if (keep) {
      j = B.inv_perm[row[t] + SI.first];
      float4 q = P.sites[j];
      H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
      dkey = H.b;
    }
    uint32_t km = __ballot_sync(FULL, keep);
    while (km) {
      uint32_t key = keep ? f2o(dkey) : 0xffffffffu;
      uint32_t mn = __reduce_min_sync(FULL, key);
      int src = __ffs(__ballot_sync(FULL, keep && key == mn)) - 1;
      PlaneT<float> Hb;
      Hb.nx = __shfl_sync(FULL, H.nx, src);
      Hb.ny = __shfl_sync(FULL, H.ny, src);
      Hb.nz = __shfl_sync(FULL, H.nz, src);
      Hb.b = __shfl_sync(FULL, H.b, src);
      Hb.e = __shfl_sync(FULL, H.e, src);
      int hj = __shfl_sync(FULL, j, src);
      if ((int)lane == src) keep = false;
      km &= ~(1u << src);
      int rc = clip_cell(c, S, Hb, hj, P.sites, false);
      if (rc == CLIP_OVERFLOW || rc == CLIP_OVF_PLANES) return false;
      if (rc == CLIP_EMPTY) return true;
    }
  }
  nv = gather_vertices(c, S, sx, sy, sz, alive);
  }
  if (B.mode == 1) {  // vertex count of the mesh output
    if (lane == 0) B.vcount[orig_i] = nv;
    return true;
  }
  if (B.mode == 2) {  // the mesh output: world positions and defining sites
    const long long base = B.voff[orig_i];
    if (base + nv > B.vcap) {
      if (lane == 0) set_error(P.st, VD_ERR_CAPACITY);
      return true;
    }
    for (int t = (int)lane; t < nv; t += 32) {
      const float4 v = S.nvp[t];
      const uint32_t T = S.nvt[t];
      B.vout[3 * (base + t)] = c.me.x + v.x;
      B.vout[3 * (base + t) + 1] = c.me.y + v.y;
      B.vout[3 * (base + t) + 2] = c.me.z + v.z;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const int id = S.pid[(T >> (8 * k)) & 255u];
        B.vsites[3 * (base + t) + k] = id >= 0 ? P.perm[id] - SI.first : id;
      }
    }
    return true;
  }
  const float cx = sx / nv, cy = sy / nv, cz = sz / nv;
  for (int f = (int)lane; f < PCAP; f += 32)
#pragma unroll
    for (int q = 0; q < 10; q++) SM.acc[f][q] = 0.f;
  __syncwarp();
  float V = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f;
  for (int it = (int)lane; it < 3 * nv; it += 32) {
    int t = it / 3, rho = it % 3;
    uint32_t T = S.nvt[t];
    uint32_t U = T | (T << 24);
    uint32_t xy = (U >> (8 * rho)) & 0xffffu;
    uint32_t fx = xy & 255u, fy = xy >> 8;
    uint32_t q = fy | (fx << 8);
    int u = 0;
    while (u < nv && !tri_has_pair(S.nvt[u], q)) u++;
    if (u >= nv) continue;
    float4 pf = S.pl[fy];
    float hgt = fmaf(pf.x, cx, fmaf(pf.y, cy, fmaf(pf.z, cz, -pf.w)));
    float g[3] = {-hgt * pf.x, -hgt * pf.y, -hgt * pf.z};
    float4 va = S.nvp[t], vb = S.nvp[u];
    float a[3] = {va.x - cx, va.y - cy, va.z - cz};
    float b[3] = {vb.x - cx, vb.y - cy, vb.z - cz};
    float det = g[0] * (a[1] * b[2] - a[2] * b[1]) + g[1] * (a[2] * b[0] - a[0] * b[2]) +
                g[2] * (a[0] * b[1] - a[1] * b[0]);
    V += det;
    Mx += det * (g[0] + a[0] + b[0]);
    My += det * (g[1] + a[1] + b[1]);
    Mz += det * (g[2] + a[2] + b[2]);
    if (S.pid[fy] < 0) continue;  // box faces do not move
    face_accumulate(SM.acc[fy], g, a, b, pf);
  }
  V = warp_sumf(V) * (1.0f / 6.0f);
  Mx = warp_sumf(Mx) * (1.0f / 24.0f);
  My = warp_sumf(My) * (1.0f / 24.0f);
  Mz = warp_sumf(Mz) * (1.0f / 24.0f);
  __syncwarp();
  if (!(V > 0.f)) return true;
  // local centroid g~ (relative to p_i) and the loss coefficients
  const float gx = cx + Mx / V, gy = cy + My / V, gz = cz + Mz / V;
  float gv = B.gvol ? B.gvol[orig_i] : 0.f;
  float d0 = 0.f, d1 = 0.f, d2 = 0.f;
  if (B.gcen) {
    d0 = B.gcen[3 * (size_t)orig_i];
    d1 = B.gcen[3 * (size_t)orig_i + 1];
    d2 = B.gcen[3 * (size_t)orig_i + 2];
  }
  const float b0 = d0 / V, b1 = d1 / V, b2 = d2 / V;
  const float ap = gv - (b0 * gx + b1 * gy + b2 * gz);
  float gpi0 = 0.f, gpi1 = 0.f, gpi2 = 0.f, gwi = 0.f;
#pragma unroll
  for (int w = 0; w < NPW; w++) {
    int f = 32 * w + (int)lane;
    if (!((alive[w] >> lane) & 1u) || S.pid[f] < 0) continue;
    int js = S.pid[f];
    face_gradient(SM.acc[f], cx, cy, cz, c.me, P.sites[js], P.perm[js], ap, b0, b1, b2, B.gp, B.gw, gpi0, gpi1,
                  gpi2, gwi);
  }
  if (B.gvert) {  // gradients of the cell's vertices (mesh order)
    const long long base = B.voff[orig_i];
    for (int t = (int)lane; t < nv; t += 32) {
      const float* g = B.gvert + 3 * (base + t);
      const float g0 = g[0], g1 = g[1], g2 = g[2];
      if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) continue;
      const uint32_t T = S.nvt[t];
      const int ids[3] = {S.pid[T & 255u], S.pid[(T >> 8) & 255u], S.pid[(T >> 16) & 255u]};
      vertex_gradient(P.sites, P.perm, c.me, S.nvp[t], ids, g0, g1, g2, B.gp, B.gw, gpi0, gpi1, gpi2, gwi);
    }
  }
  gpi0 = warp_sumf(gpi0);
  gpi1 = warp_sumf(gpi1);
  gpi2 = warp_sumf(gpi2);
  gwi = warp_sumf(gwi);
  if (lane == 0) {
    atomicAdd(&B.gp[3 * (size_t)orig_i], gpi0);
    atomicAdd(&B.gp[3 * (size_t)orig_i + 1], gpi1);
    atomicAdd(&B.gp[3 * (size_t)orig_i + 2], gpi2);
    if (B.gw) atomicAdd(&B.gw[orig_i], gwi);
  }
  __syncwarp();
  return true;
}

__device__ inline void flush_back(const BackBuffers& B, const Counters& ct, unsigned lane) {
  long long f64 = ct.fp64, f64a = ct.fp64amb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f64 += __shfl_xor_sync(FULL, f64, o);
    f64a += __shfl_xor_sync(FULL, f64a, o);
  }
  if (lane == 0) {
    if (f64) atomicAdd((unsigned long long*)&B.c.st->fp64_fallbacks, (unsigned long long)f64);
    if (f64a) atomicAdd((unsigned long long*)&B.c.st->fp64_ambiguous, (unsigned long long)f64a);
  }
}

template <int VPL, int PCAP, int QPL>
__global__ void back_kernel(BackBuffers B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BackSmem<VPL, PCAP>* Sw = reinterpret_cast<BackSmem<VPL, PCAP>*>(smem_raw);
  BackSmem<VPL, PCAP>& S = Sw[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  if (lane == 0) S.w.ct = WarpCounters{};
  __syncwarp();
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&B.work[0], 1);
    item = __shfl_sync(FULL, item, 0) + B.c.cell_begin;
    if (item >= B.c.cell_end) break;
    if (!back_cell<VPL, PCAP, QPL>(B, S, item) && lane == 0) {
      int k = atomicAdd(B.list_count, 1);
      if (k < B.list_cap)
        B.list[k] = item;
      else
        set_error(B.c.st, VD_ERR_CELL_OVERFLOW);
    }
  }
  __syncwarp();
  if (lane == 0) {
    if (S.w.ct.fp64) atomicAdd((unsigned long long*)&B.c.st->fp64_fallbacks, (unsigned long long)S.w.ct.fp64);
    if (S.w.ct.fp64amb) atomicAdd((unsigned long long*)&B.c.st->fp64_ambiguous, (unsigned long long)S.w.ct.fp64amb);
  }
}

// ---------------------------------------------------------------- large cells

// Restore the forward's polytope of large cell si from the large-cell tape
// (planes recomputed from their ids exactly as the forward computed them).
// False, with the arena untouched, if the cell has no valid record.
__device__ inline bool big_tape_read(BigCell& c, const BigArena& A, const BackBuffers& B, int si) {
  const CellBuffers& P = B.c;
  const int4 h = *reinterpret_cast<const int4*>(B.tape + (size_t)si * kTapeStride);
  if (h.x != -2 || !P.btape) return false;
  const long long off = (long long)(((unsigned long long)(unsigned)h.w << 32) | (unsigned long long)(unsigned)h.z);
  if (off < 0 || (off & 15) || off + 16 > P.btape_cap) return false;
  const char* rec = P.btape + off;
  const int4 rh = *reinterpret_cast<const int4*>(rec);
  const int nv = rh.x, npl = rh.y;
  if (nv <= 0 || nv > kBigV || npl <= 0 || npl > kBigP || npl != h.y || off + big_tape_bytes(nv, npl) > P.btape_cap)
    return false;
  const float4* vp = reinterpret_cast<const float4*>(rec + 16);
  const uint64_t* vt = reinterpret_cast<const uint64_t*>(rec + 16 + 16 * (size_t)nv);
  const int* pid = reinterpret_cast<const int*>(rec + 16 + 24 * (size_t)nv);
  const unsigned lane = lane_id();
  bool ok = true;
  for (int p = (int)lane; p < npl; p += 32) ok = ok && pid[p] >= -6 && pid[p] < P.n;
  for (int i = (int)lane; i < nv; i += 32) {
    const uint64_t T = vt[i];
    ok = ok && (int)bfield(T, 0) < npl && (int)bfield(T, 1) < npl && (int)bfield(T, 2) < npl;
  }
  if (!__all_sync(FULL, ok)) return false;
  for (int i = (int)lane; i < nv; i += 32) {
    A.vp[i] = vp[i];
    A.vt[i] = vt[i];
  }
  for (int p = (int)lane; p < npl; p += 32) {
    const int id = pid[p];
    PlaneT<float> H;
    if (id >= 0) {
      const float4 q = P.sites[id];
      H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
    } else {
      H = box_plane<float>(-1 - id, c.me.x, c.me.y, c.me.z, c.lo, c.hi);
    }
    A.pl[p] = make_float4(H.nx, H.ny, H.nz, H.b);
    A.pe[p] = H.e;
    A.pid[p] = id;
  }
  c.nv = nv;
  c.nlive = nv;
  c.nfree = 0;
  c.unsorted = 0;
  c.npl = npl;
  __syncwarp();
  return true;
}

__device__ bool big_back_cell(const BackBuffers& B, const BigArena& A, int si, Counters& ct) {
  const CellBuffers& P = B.c;
  const unsigned lane = lane_id();
  BigCell c;
  c.me = P.sites[si];
  c.fp64 = P.cfg.precision == 0;
  const int orig_i = P.perm[si];
  const int set = P.nsets > 1 ? (int)(P.keys[si] >> P.set_shift) : 0;
  const SetInfo& SI = P.sets[set];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.lo[k] = SI.lo[k];
    c.hi[k] = SI.hi[k];
  }
  const int cnt = P.counts[orig_i];
  if (cnt <= 0) return true;
  // the forward's polytope from the large-cell tape, else re-clipped from
  // the cell's neighbour row
  const bool restored = B.tape && big_tape_read(c, A, B, si);
  if (restored && lane == 0) atomicAdd((unsigned long long*)&P.st->btape_restored, 1ull);
  if (!restored) {
    big_init(c, A, 0);
    const int slot = P.ovf_slot[orig_i];
    const int* row = slot >= 0 ? P.pool + slot : P.scratch + (size_t)orig_i * P.stride;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      int t = c0 + (int)lane;
      bool keep = t < cnt;
      int j = 0;
      PlaneT<float> H;
      H.nx = H.ny = H.nz = H.b = H.e = 0.f;
      float dkey = INFINITY;
      if (keep) {
        j = B.inv_perm[row[t] + SI.first];
        float4 q = P.sites[j];
        H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
        dkey = H.b;
      }
      uint32_t km = __ballot_sync(FULL, keep);
      while (km) {
        uint32_t key = keep ? f2o(dkey) : 0xffffffffu;
        uint32_t mn = __reduce_min_sync(FULL, key);
        int src = __ffs(__ballot_sync(FULL, keep && key == mn)) - 1;
        PlaneT<float> Hb;
        Hb.nx = __shfl_sync(FULL, H.nx, src);
        Hb.ny = __shfl_sync(FULL, H.ny, src);
        Hb.nz = __shfl_sync(FULL, H.nz, src);
        Hb.b = __shfl_sync(FULL, H.b, src);
        Hb.e = __shfl_sync(FULL, H.e, src);
        int hj = __shfl_sync(FULL, j, src);
        if ((int)lane == src) keep = false;
        km &= ~(1u << src);
        int rc = big_clip(c, A, Hb, hj, P.sites, ct, false);
        if (rc == CLIP_OVERFLOW) return false;
        if (rc == CLIP_EMPTY) return true;
      }
    }
    big_compact(c, A);
  }
  if (B.mode == 1) {
    if (lane == 0) B.vcount[orig_i] = c.nv;
    return true;
  }
  if (B.mode == 2) {
    const long long base = B.voff[orig_i];
    if (base + c.nv > B.vcap) {
      if (lane == 0) set_error(P.st, VD_ERR_CAPACITY);
      return true;
    }
    for (int t = (int)lane; t < c.nv; t += 32) {
      const float4 v = A.vp[t];
      const uint64_t T = A.vt[t];
      B.vout[3 * (base + t)] = c.me.x + v.x;
      B.vout[3 * (base + t) + 1] = c.me.y + v.y;
      B.vout[3 * (base + t) + 2] = c.me.z + v.z;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const int id = A.pid[bfield(T, k)];
        B.vsites[3 * (base + t) + k] = id >= 0 ? P.perm[id] - SI.first : id;
      }
    }
    return true;
  }
  big_mark_planes(c, A);
  const uint32_t hmask = big_hash_vertices(c, A);
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = (int)lane; i < c.nv; i += 32) {
    float4 v = A.vp[i];
    sx += v.x;
    sy += v.y;
    sz += v.z;
  }
  const float cx = warp_sumf(sx) / c.nv, cy = warp_sumf(sy) / c.nv, cz = warp_sumf(sz) / c.nv;
  for (int q = (int)lane; q < 10 * c.npl; q += 32) A.acc[q] = 0.f;
  __syncwarp();
  float V = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f;
  for (int it = (int)lane; it < 3 * c.nv; it += 32) {
    int t = it / 3, rho = it % 3;
    uint32_t q = bpair(A.vt[t], rho);
    uint32_t fy = q >> 16;
    int u = hash_find(A, brev(q), hmask);
    if (u < 0) continue;
    float4 pf = A.pl[fy];
    float hgt = fmaf(pf.x, cx, fmaf(pf.y, cy, fmaf(pf.z, cz, -pf.w)));
    float g[3] = {-hgt * pf.x, -hgt * pf.y, -hgt * pf.z};
    float4 va = A.vp[t], vb = A.vp[u];
    float a[3] = {va.x - cx, va.y - cy, va.z - cz};
    float b[3] = {vb.x - cx, vb.y - cy, vb.z - cz};
    float det = g[0] * (a[1] * b[2] - a[2] * b[1]) + g[1] * (a[2] * b[0] - a[0] * b[2]) +
                g[2] * (a[0] * b[1] - a[1] * b[0]);
    V += det;
    Mx += det * (g[0] + a[0] + b[0]);
    My += det * (g[1] + a[1] + b[1]);
    Mz += det * (g[2] + a[2] + b[2]);
    if (A.pid[fy] < 0) continue;
    face_accumulate(A.acc + 10 * (size_t)fy, g, a, b, pf);
  }
  V = warp_sumf(V) * (1.0f / 6.0f);
  Mx = warp_sumf(Mx) * (1.0f / 24.0f);
  My = warp_sumf(My) * (1.0f / 24.0f);
  Mz = warp_sumf(Mz) * (1.0f / 24.0f);
  __syncwarp();
  if (!(V > 0.f)) return true;
  const float gx = cx + Mx / V, gy = cy + My / V, gz = cz + Mz / V;
  float gv = B.gvol ? B.gvol[orig_i] : 0.f;
  float d0 = 0.f, d1 = 0.f, d2 = 0.f;
  if (B.gcen) {
    d0 = B.gcen[3 * (size_t)orig_i];
    d1 = B.gcen[3 * (size_t)orig_i + 1];
    d2 = B.gcen[3 * (size_t)orig_i + 2];
  }
  const float b0 = d0 / V, b1 = d1 / V, b2 = d2 / V;
  const float ap = gv - (b0 * gx + b1 * gy + b2 * gz);
  float gpi0 = 0.f, gpi1 = 0.f, gpi2 = 0.f, gwi = 0.f;
  for (int f = (int)lane; f < c.npl; f += 32) {
    if (!A.flag[f] || A.pid[f] < 0) continue;
    int js = A.pid[f];
    face_gradient(A.acc + 10 * (size_t)f, cx, cy, cz, c.me, P.sites[js], P.perm[js], ap, b0, b1, b2, B.gp, B.gw,
                  gpi0, gpi1, gpi2, gwi);
  }
  if (B.gvert) {  // gradients of the cell's vertices (mesh order)
    const long long base = B.voff[orig_i];
    for (int t = (int)lane; t < c.nv; t += 32) {
      const float* g = B.gvert + 3 * (base + t);
      const float g0 = g[0], g1 = g[1], g2 = g[2];
      if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) continue;
      const uint64_t T = A.vt[t];
      const int ids[3] = {A.pid[bfield(T, 0)], A.pid[bfield(T, 1)], A.pid[bfield(T, 2)]};
      vertex_gradient(P.sites, P.perm, c.me, A.vp[t], ids, g0, g1, g2, B.gp, B.gw, gpi0, gpi1, gpi2, gwi);
    }
  }
  gpi0 = warp_sumf(gpi0);
  gpi1 = warp_sumf(gpi1);
  gpi2 = warp_sumf(gpi2);
  gwi = warp_sumf(gwi);
  if (lane == 0) {
    atomicAdd(&B.gp[3 * (size_t)orig_i], gpi0);
    atomicAdd(&B.gp[3 * (size_t)orig_i + 1], gpi1);
    atomicAdd(&B.gp[3 * (size_t)orig_i + 2], gpi2);
    if (B.gw) atomicAdd(&B.gw[orig_i], gwi);
  }
  __syncwarp();
  return true;
}

__global__ void big_back_kernel(BackBuffers B) {
  const unsigned lane = lane_id();
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const BigArena A = big_arena(B.c.arena, slot);
  Counters ct = {};
  const int total = min(*B.list_count, B.list_cap);
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&B.work[1], 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    if (!big_back_cell(B, A, B.list[item], ct) && lane == 0) set_error(B.c.st, VD_ERR_CELL_OVERFLOW);
  }
  flush_back(B, ct, lane);
}

cudaError_t launch_backward(const BackBuffers& b, int num_sms, cudaStream_t s) {
  const int wpb = 4;
  size_t smem = sizeof(BackSmem<4, 128>) * (size_t)wpb;
  auto kern = back_kernel<4, 128, 1>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * wpb, smem);
  if (err != cudaSuccess) return err;
  kern<<<num_sms * (occ > 0 ? occ : 1), 32 * wpb, smem, s>>>(b);
  const size_t big_smem = kBigSmemPerWarp * kBigWarpsPerBlock;
  err = cudaFuncSetAttribute(big_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
  if (err != cudaSuccess) return err;
  big_back_kernel<<<num_sms, 32 * kBigWarpsPerBlock, big_smem, s>>>(b);
  return cudaGetLastError();
}

__global__ void inverse_perm_kernel(const int* __restrict__ perm, int n, int* __restrict__ inv) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) inv[perm[k]] = k;
}

cudaError_t launch_inverse_perm(const int* perm, int n, int* inv, cudaStream_t s) {
  int blocks = min((n + 255) / 256, 4096);
  inverse_perm_kernel<<<blocks, 256, 0, s>>>(perm, n, inv);
  return cudaGetLastError();
}

}  // namespace vd
