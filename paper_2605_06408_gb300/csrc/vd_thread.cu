// vd_thread.cu -- the thread-per-cell form of the fused kernel: the paper's
// own mapping (App. A.3), one cell per thread with the polytope, the plane
// list and the best-first queue in per-thread (local) memory.
//
// Same steps and predicates as the warp-per-cell kernel: best-first
// traversal (Alg. 1) with the node bound and directional radii of Sec. 4.2,
// the candidate pre-test of Sec. 4.2.1, clipping by a half-space (App. B)
// with FP32 sign tests re-evaluated in FP64 within their error bound, plane
// garbage collection when the plane list is full (App. A.4), and the same
// outputs. A cell that outgrows the per-thread capacity goes to the
// large-cell pass like an overflowing warp-path cell. The autotuner picks
// this form or the warp form per workload.
#include "vd_big.cuh"

namespace vd {

constexpr int kTV = 64;  // vertices per cell
constexpr int kTP = 48;  // planes per cell (indices < 255; 255 = dropped)
constexpr int kTQ = 48;  // queue entries

struct TCell {
  float4 vp[kTV];  // position (local frame) and error bound
  uint32_t vt[kTV];
  float4 pl[kTP];
  float pe[kTP];
  int pid[kTP];
  float qlb[kTQ];
  int qref[kTQ];
  int qocc[kTQ];  // occupied octants | push sequence << 8
  uint32_t otri[kTV];
  float4 me;
  const float* lo;
  const float* hi;
  float alo[3], ahi[3], sc[3], srad;
  int nv, npl, qn, seq;
  bool fp64;  // FP64 re-evaluation of ambiguous predicates, vertices and volumes
};

__device__ __forceinline__ PlaneT<float> t_plane(const TCell& C, int k) {
  PlaneT<float> P;
  P.nx = C.pl[k].x;
  P.ny = C.pl[k].y;
  P.nz = C.pl[k].z;
  P.b = C.pl[k].w;
  P.e = C.pe[k];
  return P;
}

__device__ __forceinline__ float t_radius(const TCell& C, int occ, int cull) {
  return cell_radius(occ, C.alo, C.ahi, C.sc, C.srad, cull);
}

// Cell AABB (padded by the largest vertex error bound) and bounding sphere.
__device__ void t_bounds(TCell& C) {
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, em = 0.0f;
  for (int v = 0; v < C.nv; v++) {
    const float4 p = C.vp[v];
    mn[0] = fminf(mn[0], p.x);
    mn[1] = fminf(mn[1], p.y);
    mn[2] = fminf(mn[2], p.z);
    mx[0] = fmaxf(mx[0], p.x);
    mx[1] = fmaxf(mx[1], p.y);
    mx[2] = fmaxf(mx[2], p.z);
    em = fmaxf(em, p.w);
  }
  for (int k = 0; k < 3; k++) {
    C.alo[k] = mn[k] - em;
    C.ahi[k] = mx[k] + em;
    C.sc[k] = 0.5f * (C.alo[k] + C.ahi[k]);
  }
  float r2 = 0.0f;
  for (int v = 0; v < C.nv; v++) {
    const float4 p = C.vp[v];
    const float dx = p.x - C.sc[0], dy = p.y - C.sc[1], dz = p.z - C.sc[2];
    r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
  }
  C.srad = (sqrtf(r2) + em) * (1.0f + kCullPad);
}

// The box: 6 planes, 8 corners with det(n_a, n_b, n_c) > 0.
__device__ void t_init(TCell& C) {
  for (int f = 0; f < 6; f++) {
    const PlaneT<float> B = box_plane<float>(f, C.me.x, C.me.y, C.me.z, C.lo, C.hi);
    C.pl[f] = make_float4(B.nx, B.ny, B.nz, B.b);
    C.pe[f] = B.e;
    C.pid[f] = -1 - f;
  }
  for (int v = 0; v < 8; v++) {
    const int sx = v & 1, sy = (v >> 1) & 1, sz = (v >> 2) & 1;
    int a = sx, b = 2 + sy, d = 4 + sz;
    if ((sx + sy + sz) & 1) {
      const int t = b;
      b = d;
      d = t;
    }
    float x, y, z, e;
    vertex3<float>(t_plane(C, a), t_plane(C, b), t_plane(C, d), x, y, z, e);
    C.vp[v] = make_float4(x, y, z, e);
    C.vt[v] = (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)d << 16);
  }
  C.nv = 8;
  C.npl = 6;
  C.qn = 0;
  C.seq = 0;
  t_bounds(C);
}

// FP64 re-evaluation of "vertex tri lies outside the plane of site hpid".
static __device__ __noinline__ bool t_resolve64(const TCell& C, uint32_t tri, int hpid,
                                                const float4* __restrict__ sites, long long& amb) {
  const Plane64u A = plane64u(C.pid[tri & 255u], C.me, C.lo, C.hi, sites);
  const Plane64u B = plane64u(C.pid[(tri >> 8) & 255u], C.me, C.lo, C.hi, sites);
  const Plane64u D = plane64u(C.pid[(tri >> 16) & 255u], C.me, C.lo, C.hi, sites);
  const Plane64u H = plane64u(hpid, C.me, C.lo, C.hi, sites);
  bool a = false;
  const bool out = side64u(A, B, D, H, a);
  if (a) amb++;
  return out;
}

// Plane garbage collection (App. A.4): keep the planes the inside vertices
// (not in `out`) use, renumber every triplet; a dropped plane becomes 255,
// which matches no kept index (the hole walk only compares indices).
__device__ void t_gc(TCell& C, uint64_t out) {
  uint8_t map[kTP];
  uint64_t used = 0;
  for (int v = 0; v < C.nv; v++)
    if (!((out >> v) & 1ull)) {
      const uint32_t T = C.vt[v];
      used |= (1ull << (T & 255u)) | (1ull << ((T >> 8) & 255u)) | (1ull << ((T >> 16) & 255u));
    }
  int w = 0;
  for (int p = 0; p < C.npl; p++) {
    if ((used >> p) & 1ull) {
      map[p] = (uint8_t)w;
      C.pl[w] = C.pl[p];
      C.pe[w] = C.pe[p];
      C.pid[w] = C.pid[p];
      w++;
    } else {
      map[p] = 255;
    }
  }
  for (int v = 0; v < C.nv; v++) {
    const uint32_t T = C.vt[v];
    C.vt[v] = (uint32_t)map[T & 255u] | ((uint32_t)map[(T >> 8) & 255u] << 8) | ((uint32_t)map[(T >> 16) & 255u] << 16);
  }
  C.npl = w;
}

// Clip by plane H of site hpid (App. B).
__device__ int t_clip(TCell& C, const PlaneT<float>& H, int hpid, const float4* __restrict__ sites, Counters& ct) {
  uint64_t out = 0;
  int k = 0;
  for (int v = 0; v < C.nv; v++) {
    const float4 p = C.vp[v];
    const float s = side<float>(H, p.x, p.y, p.z);
    bool o = s > 0.0f;
    if (C.fp64 && ambiguous<float>(s, p.w, H.e)) {
      ct.fp64++;
      o = t_resolve64(C, C.vt[v], hpid, sites, ct.fp64amb);
    }
    if (o) {
      out |= 1ull << v;
      k++;
    }
  }
  ct.vtests += C.nv;
  if (k == 0) return CLIP_NONE;
  if (k == C.nv) return CLIP_EMPTY;
  if (C.npl >= kTP) {
    t_gc(C, out);
    if (C.npl >= kTP) return CLIP_OVF_PLANES;
  }
  const int h = C.npl++;
  C.pl[h] = make_float4(H.nx, H.ny, H.nz, H.b);
  C.pe[h] = H.e;
  C.pid[h] = hpid;
  // the outside vertices' triplets, then the inside ones compacted in place
  int w = 0, o = 0;
  for (int v = 0; v < C.nv; v++) {
    if ((out >> v) & 1ull) {
      C.otri[o++] = C.vt[v];
    } else {
      C.vp[w] = C.vp[v];
      C.vt[w] = C.vt[v];
      w++;
    }
  }
  C.nv = w;
  // hole edges: directed pairs (a,b) of outside vertices whose reverse is
  // in no other outside vertex -> new vertex (a, b, h)
  for (int t = 0; t < k; t++) {
    const uint32_t T = C.otri[t];
    const uint32_t U = T | (T << 24);
    for (int r = 0; r < 3; r++) {
      const uint32_t ab = (U >> (8 * r)) & 0xffffu;
      const uint32_t a = ab & 255u, b = ab >> 8;
      const uint32_t q = b | (a << 8);
      bool interior = false;
      for (int u = 0; u < k && !interior; u++) interior = tri_has_pair(C.otri[u], q);
      if (interior) continue;
      if (C.nv >= kTV) return CLIP_OVERFLOW;
      float x, y, z, ev;
      vertex3<float>(t_plane(C, (int)a), t_plane(C, (int)b), H, x, y, z, ev);
      if (C.fp64 && !(ev <= kRefineRel * (fabsf(x) + fabsf(y) + fabsf(z)))) {
        refine_vertex(C.pid[a], C.pid[b], hpid, C.me, C.lo, C.hi, sites, x, y, z, ev);
        ct.refv++;
      }
      C.vp[C.nv] = make_float4(x, y, z, ev);
      C.vt[C.nv] = a | (b << 8) | ((uint32_t)h << 16);
      C.nv++;
      ct.newv++;
    }
  }
  return CLIP_DONE;
}

// Sites of one leaf, in index order (the cell does not depend on the order).
__device__ int t_leaf(TCell& C, int ref, int si, int orig_i, const CellBuffers& P, Counters& ct, bool& changed) {
  const int first = leaf_first(ref), cnt = leaf_count(ref);
  for (int j = first; j < first + cnt; j++) {
    if (j == si || P.loser[j]) continue;
    const float4 q = P.sites[j];
    const float nx = q.x - C.me.x, ny = q.y - C.me.y, nz = q.z - C.me.z;
    if (nx == 0.0f && ny == 0.0f && nz == 0.0f) {
      // duplicate positions: the larger weight, then the lower index, wins
      if (q.w > C.me.w || (q.w == C.me.w && P.perm[j] < orig_i)) return CLIP_EMPTY;
      continue;
    }
    const float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    const float beta = 0.5f * (nn + (C.me.w - q.w));
    if (!candidate_test(nx, ny, nz, nn, beta, C.me.w, q.w, C.alo, C.ahi, C.sc, C.srad, P.cfg.cull_mode)) continue;
    ct.cand++;
    const PlaneT<float> H = site_plane<float>(C.me.x, C.me.y, C.me.z, C.me.w, q.x, q.y, q.z, q.w);
    const int rc = t_clip(C, H, j, P.sites, ct);
    if (rc == CLIP_EMPTY || rc == CLIP_OVERFLOW || rc == CLIP_OVF_PLANES) return rc;
    if (rc == CLIP_DONE) {
      ct.clips++;
      changed = true;
    }
  }
  return CLIP_NONE;
}

// Outputs of a finished non-empty cell. Returns false (reason set) if the
// neighbour list does not fit the cell's row.
__device__ bool t_outputs(TCell& C, const CellBuffers& P, int orig_i, int setfirst, int* row, Counters& ct,
                          int& reason) {
  // neighbours: site planes some vertex references
  uint64_t used = 0;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int v = 0; v < C.nv; v++) {
    const uint32_t T = C.vt[v];
    used |= (1ull << (T & 255u)) | (1ull << ((T >> 8) & 255u)) | (1ull << ((T >> 16) & 255u));
    sx += C.vp[v].x;
    sy += C.vp[v].y;
    sz += C.vp[v].z;
  }
  int cnt = 0;
  for (int p = 0; p < C.npl; p++)
    if (((used >> p) & 1ull) && C.pid[p] >= 0) cnt++;
  if (cnt > P.stride) {
    reason = OVF_NEIGHBORS;
    return false;
  }
  // insertion sort into the row
  int nb = 0;
  for (int p = 0; p < C.npl; p++) {
    if (!((used >> p) & 1ull) || C.pid[p] < 0) continue;
    const int val = P.perm[C.pid[p]] - setfirst;
    int t = nb++;
    while (t > 0 && row[t - 1] > val) {
      row[t] = row[t - 1];
      t--;
    }
    row[t] = val;
  }
  // volume and first moment: tetrahedra (c, g_f, a, b) for every directed
  // edge a -> b of face f, c = vertex mean, g_f = the foot of c on plane f
  const float cx = sx / C.nv, cy = sy / C.nv, cz = sz / C.nv;
  float V = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f, Sabs = 0.f, emax = 0.f;
  for (int t = 0; t < C.nv; t++) {
    const uint32_t T = C.vt[t];
    const uint32_t U = T | (T << 24);
    const float4 a4 = C.vp[t];
    emax = fmaxf(emax, a4.w);
    for (int r = 0; r < 3; r++) {
      const uint32_t xy = (U >> (8 * r)) & 0xffffu;
      const uint32_t fx = xy & 255u, fy = xy >> 8;
      const uint32_t q = fy | (fx << 8);
      int u = 0;
      while (u < C.nv && !tri_has_pair(C.vt[u], q)) u++;
      if (u >= C.nv) continue;
      const float4 pf = C.pl[fy];
      const float hgt = fmaf(pf.x, cx, fmaf(pf.y, cy, fmaf(pf.z, cz, -pf.w)));
      const float gx = -hgt * pf.x, gy = -hgt * pf.y, gz = -hgt * pf.z;
      const float4 b4 = C.vp[u];
      const float ax = a4.x - cx, ay = a4.y - cy, az = a4.z - cz;
      const float bx = b4.x - cx, by = b4.y - cy, bz = b4.z - cz;
      const float det = gx * (ay * bz - az * by) + gy * (az * bx - ax * bz) + gz * (ax * by - ay * bx);
      V += det;
      Mx += det * (gx + ax + bx);
      My += det * (gy + ay + by);
      Mz += det * (gz + az + bz);
      const float e1x = ax - gx, e1y = ay - gy, e1z = az - gz, e2x = bx - gx, e2y = by - gy, e2z = bz - gz;
      const float crx = e1y * e2z - e1z * e2y, cry = e1z * e2x - e1x * e2z, crz = e1x * e2y - e1y * e2x;
      Sabs += sqrtf(crx * crx + cry * cry + crz * crz);
    }
  }
  V *= 1.0f / 6.0f;
  Mx *= 1.0f / 24.0f;
  My *= 1.0f / 24.0f;
  Mz *= 1.0f / 24.0f;
  Sabs *= 0.5f;
  float L = 0.f;
  for (int k = 0; k < 3; k++) L += fmaxf(C.alo[k] * C.alo[k], C.ahi[k] * C.ahi[k]);
  L = sqrtf(L);
  double ox = cx, oy = cy, oz = cz, Vd = V;
  if (C.fp64 && volume_needs_fp64(V, L, Sabs, emax)) {
    // FP64: vertices re-solved from the inputs; each face's fan anchored at
    // its lowest-index vertex
    ct.refvol++;
    double vd[3 * kTV];
    int anchor[kTP];
    for (int p = 0; p < C.npl; p++) anchor[p] = 0x7fffffff;
    for (int t = 0; t < C.nv; t++) {
      const uint32_t T = C.vt[t];
      double x, y, z;
      vertex64(T & 255u, (T >> 8) & 255u, (T >> 16) & 255u, C.pid, C.me, C.lo, C.hi, P.sites, x, y, z);
      vd[3 * t] = x - cx;
      vd[3 * t + 1] = y - cy;
      vd[3 * t + 2] = z - cz;
      for (int r = 0; r < 3; r++) {
        const int f = (int)((T >> (8 * r)) & 255u);
        anchor[f] = min(anchor[f], t);
      }
    }
    double W = 0.0, X = 0.0, Y = 0.0, Z = 0.0;
    for (int t = 0; t < C.nv; t++) {
      const uint32_t T = C.vt[t];
      const uint32_t U = T | (T << 24);
      for (int r = 0; r < 3; r++) {
        const uint32_t xy = (U >> (8 * r)) & 0xffffu;
        const uint32_t fx = xy & 255u, fy = xy >> 8;
        const uint32_t q = fy | (fx << 8);
        int u = 0;
        while (u < C.nv && !tri_has_pair(C.vt[u], q)) u++;
        const int g = anchor[fy];
        if (u >= C.nv || g == t || g == u) continue;
        const double* A = &vd[3 * g];
        const double* B = &vd[3 * t];
        const double* D = &vd[3 * u];
        const double det = A[0] * (B[1] * D[2] - B[2] * D[1]) + A[1] * (B[2] * D[0] - B[0] * D[2]) +
                           A[2] * (B[0] * D[1] - B[1] * D[0]);
        W += det;
        X += det * (A[0] + B[0] + D[0]);
        Y += det * (A[1] + B[1] + D[1]);
        Z += det * (A[2] + B[2] + D[2]);
      }
    }
    Vd = W / 6.0;
    if (Vd > 0.0) {
      ox += X / 24.0 / Vd;
      oy += Y / 24.0 / Vd;
      oz += Z / 24.0 / Vd;
    }
  } else if (V > 0.0f) {
    ox += Mx / V;
    oy += My / V;
    oz += Mz / V;
  }
  P.counts[orig_i] = cnt;
  P.vol[orig_i] = (float)Vd;
  P.cen[3 * (size_t)orig_i] = (float)((double)C.me.x + ox);
  P.cen[3 * (size_t)orig_i + 1] = (float)((double)C.me.y + oy);
  P.cen[3 * (size_t)orig_i + 2] = (float)((double)C.me.z + oz);
  return true;
}

__device__ bool t_push(TCell& C, float lb, int ref, int occ) {
  if (C.qn >= kTQ) return false;
  C.qlb[C.qn] = lb;
  C.qref[C.qn] = ref;
  C.qocc[C.qn] = occ | (C.seq << 8);
  C.qn++;
  C.seq++;
  return true;
}

// Pop the best entry still valid under the current bounds (Alg. 1
// backtracking); entries that fail the re-test are dropped.
__device__ bool t_pop(TCell& C, int cull, int trav, int& ref) {
  int live = 0, best = -1;
  float bestk = INFINITY;
  for (int i = 0; i < C.qn; i++) {
    const float lb = C.qlb[i];
    const int oc = C.qocc[i];
    const float R = t_radius(C, oc & 63, cull);
    if (cull != 2 && lb > R * (1.0f + kCullPad)) continue;
    const float key = trav == 0 ? lb - R : -(float)(oc >> 8);
    C.qlb[live] = lb;
    C.qref[live] = C.qref[i];
    C.qocc[live] = oc;
    if (best < 0 || key < bestk) {
      bestk = key;
      best = live;
    }
    live++;
  }
  C.qn = live;
  if (best < 0) return false;
  ref = C.qref[best];
  C.qn--;
  C.qlb[best] = C.qlb[C.qn];
  C.qref[best] = C.qref[C.qn];
  C.qocc[best] = C.qocc[C.qn];
  return true;
}

// Build one cell; false = overflow (reason set).
__device__ bool t_build_cell(const CellBuffers& P, int si, Counters& ct, long long& empties, int& reason) {
  const int orig_i = P.perm[si];
  const float4 me = P.sites[si];
  if (P.loser[si]) {
    P.counts[orig_i] = 0;
    P.vol[orig_i] = 0.0f;
    P.cen[3 * (size_t)orig_i] = me.x;
    P.cen[3 * (size_t)orig_i + 1] = me.y;
    P.cen[3 * (size_t)orig_i + 2] = me.z;
    empties++;
    return true;
  }
  const int set = P.nsets > 1 ? (int)(P.keys[si] >> P.set_shift) : 0;
  const SetInfo& SI = P.sets[set];
  TCell C;
  C.me = me;
  C.fp64 = P.cfg.precision == 0;
  C.lo = SI.lo;
  C.hi = SI.hi;
  t_init(C);
  const int cull = P.cfg.cull_mode, trav = P.cfg.traversal;
  bool empty = false;
  int cur = SI.root;
  bool have = true;
  while (true) {
    if (have) {
      if (ref_is_leaf(cur)) {
        bool changed = false;
        const int rc = t_leaf(C, cur, si, orig_i, P, ct, changed);
        if (rc == CLIP_EMPTY) {
          empty = true;
          break;
        }
        if (rc == CLIP_OVERFLOW || rc == CLIP_OVF_PLANES) {
          reason = rc == CLIP_OVERFLOW ? OVF_VERTICES : OVF_PLANES;
          return false;
        }
        if (changed) t_bounds(C);
        have = false;
      } else {
        const float4* nd = P.nodes + 4 * (size_t)cur;
        const float4 lo0 = __ldg(nd), hi0 = __ldg(nd + 1), lo1 = __ldg(nd + 2), hi1 = __ldg(nd + 3);
        auto rad = [&](int o) { return t_radius(C, o, cull); };
        float lb0, lb1, key0, key1;
        int occ0, occ1;
        const bool k0 = node_test_r(lo0, hi0, C.me, rad, cull, lb0, occ0, key0);
        const bool k1 = node_test_r(lo1, hi1, C.me, rad, cull, lb1, occ1, key1);
        const int r0 = __float_as_int(hi0.w), r1 = __float_as_int(hi1.w);
        ct.nodes += 2;
        if (k0 && k1) {
          const bool near0 = key0 <= key1;  // nearer child first (both traversals)
          cur = near0 ? r0 : r1;
          if (!t_push(C, near0 ? lb1 : lb0, near0 ? r1 : r0, near0 ? occ1 : occ0)) {
            reason = OVF_QUEUE;
            return false;
          }
        } else if (k0) {
          cur = r0;
        } else if (k1) {
          cur = r1;
        } else {
          have = false;
        }
      }
      if (have) continue;
    }
    if (!t_pop(C, cull, trav, cur)) break;
    have = true;
  }
  if (empty) {
    P.counts[orig_i] = 0;
    P.vol[orig_i] = 0.0f;
    P.cen[3 * (size_t)orig_i] = me.x;
    P.cen[3 * (size_t)orig_i + 1] = me.y;
    P.cen[3 * (size_t)orig_i + 2] = me.z;
    empties++;
    return true;
  }
  int* row = P.scratch + (size_t)orig_i * P.stride;
  return t_outputs(C, P, orig_i, SI.first, row, ct, reason);
}

__global__ void __launch_bounds__(128) cells_thread_kernel(CellBuffers P) {
  const unsigned lane = lane_id();
  Counters ct = {};
  long long empties = 0, overflows = 0;
  long long reasons[4] = {0, 0, 0, 0};
  while (true) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&P.work[0], 32);
    base = __shfl_sync(FULL, base, 0) + P.cell_begin;
    if (base >= P.cell_end) break;
    const int si = base + (int)lane;
    if (si < P.cell_end) {
      int reason = 0;
      const long long amb0 = ct.fp64amb;
      const bool built = t_build_cell(P, si, ct, empties, reason);
      if (ct.fp64amb != amb0) record_ambiguous(P.st, P.amb_list, P.amb_cap, P.perm[si]);
      if (!built) {
        overflows++;
        reasons[reason]++;
        const int orig = P.perm[si];
        const int slot = atomicAdd(&P.st->ovf_count, 1);
        if (slot < P.ovf_cap) {
          P.ovf_list[slot] = si;
        } else {
          P.counts[orig] = 0;
          P.vol[orig] = __int_as_float(0x7fc00000);
          set_error(P.st, VD_ERR_CELL_OVERFLOW);
        }
      }
    }
  }
  // per-thread tallies: reduce over the warp, lane 0 publishes
  long long vals[15] = {ct.cand, ct.clips, ct.nodes, ct.vtests, ct.newv, ct.fp64, ct.fp64amb, ct.refv, ct.refvol,
                        empties, overflows, reasons[0], reasons[1], reasons[2], reasons[3]};
#pragma unroll
  for (int k = 0; k < 15; k++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vals[k] += __shfl_xor_sync(FULL, vals[k], o);
  if (lane == 0) {
    if (vals[9]) atomicAdd((unsigned long long*)&P.st->empty_cells, (unsigned long long)vals[9]);
    if (vals[10]) atomicAdd((unsigned long long*)&P.st->overflow_cells, (unsigned long long)vals[10]);
    for (int r = 0; r < 4; r++)
      if (vals[11 + r]) atomicAdd((unsigned long long*)&P.st->ovf_reason[r], (unsigned long long)vals[11 + r]);
    if (vals[5]) atomicAdd((unsigned long long*)&P.st->fp64_fallbacks, (unsigned long long)vals[5]);
    if (vals[6]) atomicAdd((unsigned long long*)&P.st->fp64_ambiguous, (unsigned long long)vals[6]);
    if (vals[7]) atomicAdd((unsigned long long*)&P.st->refined_vertices, (unsigned long long)vals[7]);
    if (vals[8]) atomicAdd((unsigned long long*)&P.st->refined_volumes, (unsigned long long)vals[8]);
    if (P.cfg.counters) {
      atomicAdd((unsigned long long*)&P.st->candidates, (unsigned long long)vals[0]);
      atomicAdd((unsigned long long*)&P.st->clips, (unsigned long long)vals[1]);
      atomicAdd((unsigned long long*)&P.st->nodes, (unsigned long long)vals[2]);
      atomicAdd((unsigned long long*)&P.st->vertex_tests, (unsigned long long)vals[3]);
      atomicAdd((unsigned long long*)&P.st->new_vertices, (unsigned long long)vals[4]);
    }
  }
}

cudaError_t launch_cells_thread(const CellBuffers& c, int num_sms, cudaStream_t s) {
  int per_sm = c.cfg.blocks_per_sm;
  if (per_sm <= 0) {
    int occ = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cells_thread_kernel, 128, 0);
    if (err != cudaSuccess) return err;
    per_sm = occ > 0 ? occ : 1;
  }
  cells_thread_kernel<<<num_sms * per_sm, 128, 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace vd
