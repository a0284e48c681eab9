// vd_cells.cu -- the fused per-cell kernel: best-first BVH traversal (Alg. 1),
// directional and node culling (Sec. 4.2), convex cell clipping (Sec. 4.1,
// App. B), neighbour extraction and volume/centroid.
//
// GB300 mapping (differs from the paper's thread-per-cell design, App. A):
// one warp per cell in a persistent grid that pulls cells from a global
// counter in Morton order. The polytope's vertices live in registers
// (VPL slots per lane, position + error bound + plane triplet), its planes
// in shared memory; leaf sites are loaded with one coalesced float4 per lane
// and pre-culled in parallel; the priority queue holds QPL entries per lane
// and pops its minimum with one redux.sync.
//
// A clip by plane h (App. B) classifies all vertices in parallel, collects
// the outside ones, and finds the boundary of the hole as the directed
// plane pairs (a,b) of outside vertices whose reverse pair (b,a) belongs to
// no other outside vertex; every such pair becomes the new vertex (a,b,h).
// This reaches the same polytope as the paper's sequential walk around the
// hole, in a form that runs on 32 lanes at once.
//
// Predicates run in FP32; a sign test whose value is within its error
// bound of zero is re-evaluated in FP64 from the original inputs.
#include <functional>

#include "vd_big.cuh"

namespace vd {

// GEN: the generic instantiation, which reads the ablation modes (culling,
// traversal), the event counters and the precision mode from the
// configuration; the default one (GEN = false) has them folded to
// directional culling, best-first order, no counters and mixed precision, so
// that code a timed build never runs stays out of its instruction stream
// (measured on one GB300: 7-8% faster than one kernel for both).
template <bool GEN>
struct Knobs {
  int cull, trav;
  bool counters;
  __device__ __forceinline__ explicit Knobs(const vd_config& g)
      : cull(GEN ? g.cull_mode : 0), trav(GEN ? g.traversal : 0), counters(GEN && g.counters != 0) {}
};

// Process the sites of one leaf: pre-cull all of them in parallel, then
// clip with the survivors in ascending power distance d_ij (Eq. 2).
template <int VPL, int PCAP, int QPL, bool GEN>
__device__ int process_leaf(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP, QPL>& S, int ref, int si, int orig_i,
                            const CellBuffers& P, int skip0, int skip1) {
  const unsigned lane = lane_id();
  const Knobs<GEN> K(P.cfg);
  const bool counters = K.counters;
  int j;
  bool act;
  if (ref == kKnnLeaf) {  // the KNN warm start: the cell's nearest sites
    j = (int)lane < kKnn ? S.knn[lane] : -1;
    act = j >= 0;
  } else {
    const int first = leaf_first(ref), cnt = leaf_count(ref);
    j = first + (int)lane;
    // sites of the warm-start window [skip0, skip1) were clipped already
    act = (int)lane < cnt && j != si && (j < skip0 || j >= skip1);
    if (P.cfg.warm_start == 2) {  // and so were the KNN sites
#pragma unroll
      for (int k = 0; k < kKnn; k++) act = act && S.knn[k] != j;
    }
  }
  // the site and its duplicate-loser flag are loaded together (both
  // indices are valid when act holds); a loser takes no part
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  unsigned char lost = 0;
  if (act) {
    lost = P.loser[j];
    q = P.sites[j];
  }
  act = act && lost == 0;
  PlaneT<float> H;
  H.nx = H.ny = H.nz = H.b = H.e = 0.0f;
  bool keep = false, dup = false;
  float dkey = INFINITY;
  if (act) {
    float nx = q.x - c.me.x, ny = q.y - c.me.y, nz = q.z - c.me.z;
    float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    dup = nx == 0.0f && ny == 0.0f && nz == 0.0f;
    if (!dup) {
      float beta = 0.5f * (nn + (c.me.w - q.w));
      keep = candidate_test(nx, ny, nz, nn, beta, c.me.w, q.w, c.alo, c.ahi, c.sc, c.srad, K.cull);
      if (keep) {
        H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
        dkey = H.b;
      }
    }
  }
  // duplicate positions: the larger weight, then the lower index, wins
  if (__any_sync(FULL, dup)) {
    bool beats = dup && (q.w > c.me.w || (q.w == c.me.w && P.perm[j] < orig_i));
    if (__any_sync(FULL, beats)) return CLIP_EMPTY;
  }
  uint32_t km = __ballot_sync(FULL, keep);
  if (counters && lane == 0) S.ct.cand += __popc(km);
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
    const int hj = __shfl_sync(FULL, j, src);
    if ((int)lane == src) keep = false;
    km &= ~(1u << src);
    int rc = clip_cell(c, S, Hb, hj, P.sites, counters);
    if (rc == CLIP_EMPTY || rc == CLIP_OVERFLOW || rc == CLIP_OVF_PLANES) return rc;
    if (rc == CLIP_DONE) {
      c.dirty = true;
      if (counters && lane == 0) S.ct.clips++;
    }
  }
  return CLIP_NONE;
}

// Where the outputs of a cell go (cell_outputs).
struct CellOut {
  const int* perm;
  int* counts;
  float* vol;
  float* cen;
  char* tape;
  const float4* sites;
  int stride, si, orig_i, setfirst;
  int* row;
  float4 me;
  const float* box;
  float L;  // largest distance of the cell's AABB corners from the site
  bool fp64;
};

// The cell's record for the adjoint (tape): its vertices with plane indices
// renumbered to the alive planes' order, and those planes' ids; a header of
// -1 vertices when the cell does not fit a record. Out of line, like
// cell_outputs: code that a build without a tape never runs stays out of
// the once-per-cell path.
template <int VPL, int PCAP, int QPL>
static __device__ __noinline__ void write_tape(WarpSmem<VPL, PCAP, QPL>& S, char* rec, const int nv, uint32_t a0,
                                               uint32_t a1, uint32_t a2, uint32_t a3) {
  constexpr int NPW = PCAP / 32;
  const unsigned lane = lane_id();
  const uint32_t al[4] = {a0, a1, a2, a3};
  uint32_t alive[NPW];
  int pre[NPW], nf = 0;
#pragma unroll
  for (int w = 0; w < NPW; w++) {
    alive[w] = al[w];
    pre[w] = nf;
    nf += __popc(alive[w]);
  }
  const bool fits = nv <= kTapeV && nf <= kTapeF;
  if (fits) {
    auto rank = [&](uint32_t f) -> uint32_t {
      uint32_t r = 0;
#pragma unroll
      for (int w = 0; w < NPW; w++)
        if ((f >> 5) == (uint32_t)w) r = (uint32_t)pre[w] + __popc(alive[w] & ((1u << (f & 31u)) - 1u));
      return r;
    };
    float4* tv = reinterpret_cast<float4*>(rec + kTapeVOff);
#pragma unroll 1
    for (int t = (int)lane; t < nv; t += 32) {
      const uint32_t T = S.nvt[t];
      const uint32_t R = rank(T & 255u) | (rank((T >> 8) & 255u) << 8) | (rank((T >> 16) & 255u) << 16);
      const float4 p = S.nvp[t];
      tv[t] = make_float4(p.x, p.y, p.z, __uint_as_float(R));
    }
    int* tf = reinterpret_cast<int*>(rec + kTapeFOff);
#pragma unroll
    for (int w = 0; w < NPW; w++) {
      const int f = 32 * w + (int)lane;
      if ((alive[w] >> lane) & 1u) tf[rank((uint32_t)f)] = S.pid[f];
    }
  }
  if (lane == 0) *reinterpret_cast<int4*>(rec) = make_int4(fits ? nv : -1, nf, 0, 0);
}

// The outputs of a finished cell from its vertices gathered in S (slot
// order, nv of them, coordinate sums sx, sy, sz, alive planes a0..a3): the
// neighbour row, the tape record, volume and centroid. Out of line: it runs
// once per cell, and keeping it out of the traversal loop's code helps the
// instruction cache. For the same reason its loops stay rolled and its cold
// branches (the tape, the FP64 volume) are calls: every kilobyte of code
// here measurably slows the whole kernel. Returns false, writing nothing, if
// the neighbour list is longer than a row.
template <int VPL, int PCAP, int QPL>
static __device__ __noinline__ bool cell_outputs(WarpSmem<VPL, PCAP, QPL>& S, const CellOut O, const int nv,
                                                 const float sx, const float sy, const float sz, uint32_t a0,
                                                 uint32_t a1, uint32_t a2, uint32_t a3) {
  constexpr int NPW = PCAP / 32;
  const unsigned lane = lane_id(), lt = lanemask_lt();
  const uint32_t al[4] = {a0, a1, a2, a3};
  uint32_t alive[NPW];
#pragma unroll
  for (int w = 0; w < NPW; w++) alive[w] = al[w];
  const int si = O.si, orig_i = O.orig_i;
  int* row = O.row;
  // neighbours: site planes that carry a face
  int nvals = 0;
  const int setfirst = O.setfirst;
#pragma unroll
  for (int w = 0; w < NPW; w++) {
    int f = 32 * w + (int)lane;
    bool isn = ((alive[w] >> lane) & 1u) && S.pid[f] >= 0;
    uint32_t mk = __ballot_sync(FULL, isn);
    if (isn) S.otri[nvals + __popc(mk & lt)] = (uint32_t)(O.perm[S.pid[f]] - setfirst);
    nvals += __popc(mk);
  }
  __syncwarp();
  if (nvals > O.stride) return false;  // more neighbours than a fast-path row holds
#pragma unroll 1
  for (int t = (int)lane; t < nvals; t += 32) {
    int v = (int)S.otri[t];
    int rank = 0;
#pragma unroll 1
    for (int u = 0; u < nvals; u++) rank += (int)S.otri[u] < v;
    row[rank] = v;
  }
  if (O.tape) write_tape<VPL, PCAP, QPL>(S, O.tape + (size_t)si * kTapeStride, nv, a0, a1, a2, a3);
  // volume and first moment: tetrahedra (c, g_f, v, w) for every directed
  // edge v -> w of face f (w = the other end of the edge), g_f = the foot of
  // c on plane f; c = vertex mean
  float cx = sx / nv, cy = sy / nv, cz = sz / nv;
  float V = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f, Sabs = 0.f, emax = 0.f;
#pragma unroll 1
  for (int it = (int)lane; it < 3 * nv; it += 32) {
    int t = it / 3, rho = it % 3;
    uint32_t T = S.nvt[t];
    uint32_t U = T | (T << 24);
    uint32_t xy = (U >> (8 * rho)) & 0xffffu;
    uint32_t fx = xy & 255u, fy = xy >> 8;
    uint32_t q = fy | (fx << 8);
    int u = 0;
    while (u < nv && !tri_has_pair(S.nvt[u], q)) u++;
    if (u >= nv) continue;  // cannot happen for a closed polytope
    float4 pf = S.pl[fy];
    float hgt = fmaf(pf.x, cx, fmaf(pf.y, cy, fmaf(pf.z, cz, -pf.w)));
    float gx = -hgt * pf.x, gy = -hgt * pf.y, gz = -hgt * pf.z;  // g_f - c
    float4 a = S.nvp[t], b = S.nvp[u];
    float ax = a.x - cx, ay = a.y - cy, az = a.z - cz;
    float bx = b.x - cx, by = b.y - cy, bz = b.z - cz;
    float det = gx * (ay * bz - az * by) + gy * (az * bx - ax * bz) + gz * (ax * by - ay * bx);
    V += det;
    Mx += det * (gx + ax + bx);
    My += det * (gy + ay + by);
    Mz += det * (gz + az + bz);
    float e1x = ax - gx, e1y = ay - gy, e1z = az - gz, e2x = bx - gx, e2y = by - gy, e2z = bz - gz;
    float crx = e1y * e2z - e1z * e2y, cry = e1z * e2x - e1x * e2z, crz = e1x * e2y - e1y * e2x;
    Sabs += sqrtf(crx * crx + cry * cry + crz * crz);
    emax = fmaxf(emax, a.w);
  }
  V = warp_sumf(V) * (1.0f / 6.0f);
  Mx = warp_sumf(Mx) * (1.0f / 24.0f);
  My = warp_sumf(My) * (1.0f / 24.0f);
  Mz = warp_sumf(Mz) * (1.0f / 24.0f);
  Sabs = warp_sumf(Sabs) * 0.5f;
  emax = warp_maxf(emax);
  const float L = O.L;
  double ox = cx, oy = cy, oz = cz;
  double Vd = V;
  if (O.fp64 && volume_needs_fp64(V, L, Sabs, emax)) {
    double Mxd, Myd, Mzd;
    volume_fp64(S, nv, O.me, O.box, O.box + 3, O.sites, (double)cx, (double)cy, (double)cz, Vd, Mxd, Myd, Mzd);
    if (Vd > 0.0) {
      const double iv = 1.0 / Vd;
      ox += Mxd * iv;
      oy += Myd * iv;
      oz += Mzd * iv;
    }
    if (lane == 0) S.ct.refvol++;
  } else if (V > 0.0f) {
    ox += Mx / V;
    oy += My / V;
    oz += Mz / V;
  }
  if (lane == 0) {
    O.counts[orig_i] = nvals;
    O.vol[orig_i] = (float)Vd;
    O.cen[3 * (size_t)orig_i] = (float)((double)O.me.x + ox);
    O.cen[3 * (size_t)orig_i + 1] = (float)((double)O.me.y + oy);
    O.cen[3 * (size_t)orig_i + 2] = (float)((double)O.me.z + oz);
  }
  __syncwarp();
  return true;
}

// Build one cell and write its outputs. Returns false on overflow.
template <int VPL, int PCAP, int QPL, bool GEN>
__device__ bool build_cell(const CellBuffers& P, WarpSmem<VPL, PCAP, QPL>& S, int si, int* row, long long& empties,
                           int& reason) {
  using C = Cell<VPL, PCAP, QPL>;
  constexpr int NPW = C::NPW;
  const unsigned lane = lane_id(), lt = lanemask_lt();
  const Knobs<GEN> K(P.cfg);
  const bool counters = K.counters;
  C c;
  c.me = P.sites[si];
  c.fp64 = GEN ? P.cfg.precision == 0 : true;
  const int orig_i = P.perm[si];
  if (P.loser[si]) {  // an exact duplicate site owns this position
    if (lane == 0) {
      P.counts[orig_i] = 0;
      P.vol[orig_i] = 0.0f;
      P.cen[3 * (size_t)orig_i] = c.me.x;
      P.cen[3 * (size_t)orig_i + 1] = c.me.y;
      P.cen[3 * (size_t)orig_i + 2] = c.me.z;
    }
    empties++;
    return true;
  }
  const int set = P.nsets > 1 ? (int)(P.keys[si] >> P.set_shift) : 0;
  const SetInfo& SI = P.sets[set];
  c.box = SI.lo;
  const int cull = K.cull, trav = K.trav;
  init_cell(c, S, cull);
  bool empty = false, overflow = false;

  // ---- warm start (App. A.6, with the 32 Morton-order neighbours of the
  // site instead of a KNN query: one coalesced load, no extra pass): the
  // window is the first leaf the loop below processes (one inlined copy of
  // the leaf and clip code serves both)
  int skip0 = 0, skip1 = 0;
  bool warm = P.cfg.warm_start != 0;
  int cur = SI.root;
  if (P.cfg.warm_start == 2) {  // KNN warm start (App. A.6): the list of this cell
    if (lane < kKnn) S.knn[lane] = P.knn[(size_t)si * kKnn + lane];
    __syncwarp();
    cur = kKnnLeaf;
  } else if (warm) {
    const int lo = SI.first, hi = SI.first + SI.count;
    skip0 = max(lo, min(si - 16, hi - 32));
    skip1 = min(hi, skip0 + 32);
    cur = make_leaf_ref(skip0, skip1 - skip0);
  }

  // ---- best-first traversal (Alg. 1)
  bool have = !empty;
  while (!empty) {
    if (have) {
      if (ref_is_leaf(cur)) {
        int rc = process_leaf<VPL, PCAP, QPL, GEN>(c, S, cur, si, orig_i, P, warm ? 0 : skip0, warm ? 0 : skip1);
        if (rc == CLIP_EMPTY) {
          empty = true;
          break;
        }
        if (rc == CLIP_OVERFLOW || rc == CLIP_OVF_PLANES) {
          reason = rc == CLIP_OVERFLOW ? OVF_VERTICES : OVF_PLANES;
          overflow = true;
          break;
        }
        if (c.dirty) {
          recompute_aabb(c, S, cull);
          c.dirty = false;
        }
        if (warm) {  // the warm-start window done: now the traversal from the root
          warm = false;
          cur = SI.root;
          continue;
        }
        have = false;
      } else {
        const float4* nd = P.nodes + 4 * (size_t)cur;
        float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < 4) rec = __ldg(nd + lane);
        float4 hi;
        hi.x = __shfl_down_sync(FULL, rec.x, 1);
        hi.y = __shfl_down_sync(FULL, rec.y, 1);
        hi.z = __shfl_down_sync(FULL, rec.z, 1);
        hi.w = __shfl_down_sync(FULL, rec.w, 1);
        float lb = 0.f, key = 0.f;
        int occ = 0;
        bool keep = false;
        if (lane == 0 || lane == 2) keep = node_test(rec, hi, c.me, S.rtab, cull, lb, occ, key);
        int myref = __float_as_int(hi.w);
        bool k0 = __shfl_sync(FULL, keep, 0), k1 = __shfl_sync(FULL, keep, 2);
        float key0 = __shfl_sync(FULL, key, 0), key1 = __shfl_sync(FULL, key, 2);
        int r0 = __shfl_sync(FULL, myref, 0), r1 = __shfl_sync(FULL, myref, 2);
        if (counters && lane == 0) S.ct.nodes += 2;
        if (k0 && k1) {
          bool near0 = key0 <= key1;  // nearer child first (both traversals)
          int fsrc = near0 ? 2 : 0;
          float flb = __shfl_sync(FULL, lb, fsrc);
          int focc = __shfl_sync(FULL, occ, fsrc);
          cur = near0 ? r0 : r1;
          if (!queue_push(c, S, flb, near0 ? r1 : r0, focc)) {
            reason = OVF_QUEUE;
            overflow = true;
            break;
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
    if (!queue_pop(c, S, cull, trav, cur)) break;
    have = true;
  }
  if (overflow) return false;

  float* vol = P.vol;
  float* cen = P.cen;
  if (empty) {
    if (lane == 0) {
      P.counts[orig_i] = 0;
      vol[orig_i] = 0.0f;
      cen[3 * (size_t)orig_i] = c.me.x;
      cen[3 * (size_t)orig_i + 1] = c.me.y;
      cen[3 * (size_t)orig_i + 2] = c.me.z;
    }
    empties++;
    return true;
  }

  // ---- outputs: vertex list, neighbours, volume and centroid
  float sx, sy, sz;
  uint32_t alive[NPW];
  const int nv = gather_vertices(c, S, sx, sy, sz, alive);
  float L = 0.f;
#pragma unroll
  for (int k = 0; k < 3; k++) L += fmaxf(c.alo[k] * c.alo[k], c.ahi[k] * c.ahi[k]);
  CellOut O;
  O.perm = P.perm;
  O.counts = P.counts;
  O.vol = P.vol;
  O.cen = P.cen;
  O.tape = P.tape;
  O.sites = P.sites;
  O.stride = P.stride;
  O.si = si;
  O.orig_i = orig_i;
  O.setfirst = SI.first;
  O.row = row;
  O.me = c.me;
  O.box = c.box;
  O.L = sqrtf(L);
  O.fp64 = c.fp64;
  uint32_t al[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int w = 0; w < NPW; w++) al[w] = alive[w];
  if (!cell_outputs<VPL, PCAP, QPL>(S, O, nv, sx, sy, sz, al[0], al[1], al[2], al[3])) {
    reason = OVF_NEIGHBORS;
    return false;
  }
  return true;
}

__device__ inline void flush_counters(const CellBuffers& P, const Counters& ct, unsigned lane, long long empties,
                                      long long overflows, long long failed) {
  if (lane == 0) {
    if (empties) atomicAdd((unsigned long long*)&P.st->empty_cells, (unsigned long long)empties);
    if (overflows) atomicAdd((unsigned long long*)&P.st->overflow_cells, (unsigned long long)overflows);
    if (failed) atomicAdd((unsigned long long*)&P.st->failed_cells, (unsigned long long)failed);
  }
  // FP64 re-evaluations happen on individual lanes
  long long f64 = ct.fp64, f64a = ct.fp64amb, rv = ct.refv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f64 += __shfl_xor_sync(FULL, f64, o);
    f64a += __shfl_xor_sync(FULL, f64a, o);
    rv += __shfl_xor_sync(FULL, rv, o);
  }
  if (lane == 0) {
    if (f64) atomicAdd((unsigned long long*)&P.st->fp64_fallbacks, (unsigned long long)f64);
    if (f64a) atomicAdd((unsigned long long*)&P.st->fp64_ambiguous, (unsigned long long)f64a);
    if (rv) atomicAdd((unsigned long long*)&P.st->refined_vertices, (unsigned long long)rv);
    if (ct.refvol) atomicAdd((unsigned long long*)&P.st->refined_volumes, (unsigned long long)ct.refvol);
    if (P.cfg.counters) {  // the large-cell pass counts apart from the main pass
      atomicAdd((unsigned long long*)&P.st->large_candidates, (unsigned long long)ct.cand);
      atomicAdd((unsigned long long*)&P.st->large_clips, (unsigned long long)ct.clips);
      atomicAdd((unsigned long long*)&P.st->large_nodes, (unsigned long long)ct.nodes);
      atomicAdd((unsigned long long*)&P.st->large_vtests, (unsigned long long)ct.vtests);
      atomicAdd((unsigned long long*)&P.st->large_newv, (unsigned long long)ct.newv);
    }
  }
}

__device__ inline void flush_warp_counters(const CellBuffers& P, const WarpCounters& w, unsigned lane,
                                           long long empties, long long overflows) {
  if (lane != 0) return;
  if (empties) atomicAdd((unsigned long long*)&P.st->empty_cells, (unsigned long long)empties);
  if (overflows) atomicAdd((unsigned long long*)&P.st->overflow_cells, (unsigned long long)overflows);
  if (w.fp64) atomicAdd((unsigned long long*)&P.st->fp64_fallbacks, (unsigned long long)w.fp64);
  if (w.fp64amb) atomicAdd((unsigned long long*)&P.st->fp64_ambiguous, (unsigned long long)w.fp64amb);
  if (w.refv) atomicAdd((unsigned long long*)&P.st->refined_vertices, (unsigned long long)w.refv);
  if (w.refvol) atomicAdd((unsigned long long*)&P.st->refined_volumes, (unsigned long long)w.refvol);
  if (P.cfg.counters) {
    atomicAdd((unsigned long long*)&P.st->candidates, w.cand);
    atomicAdd((unsigned long long*)&P.st->clips, w.clips);
    atomicAdd((unsigned long long*)&P.st->nodes, w.nodes);
    atomicAdd((unsigned long long*)&P.st->vertex_tests, w.vtests);
    atomicAdd((unsigned long long*)&P.st->new_vertices, w.newv);
  }
}

// VD_CELLS_MIN_BLOCKS (build option): minimum resident 256-thread blocks per
// SM the compiler must allow for, i.e. a register cap. 2 (128 registers)
// measured fastest on GB300 (mixture1M: 65.7 ms vs 74.4 ms uncapped, 93 ms
// at 3 blocks / 85 registers, which spills); 0 removes the cap.
#ifndef VD_CELLS_MIN_BLOCKS
#define VD_CELLS_MIN_BLOCKS 2
#endif
#if VD_CELLS_MIN_BLOCKS > 0
#define VD_CELLS_BOUNDS __launch_bounds__(256, VD_CELLS_MIN_BLOCKS)
#else
#define VD_CELLS_BOUNDS
#endif
template <int VPL, int PCAP, int QPL, bool GEN>
__global__ void VD_CELLS_BOUNDS cells_kernel(CellBuffers P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<VPL, PCAP, QPL>* Sw = reinterpret_cast<WarpSmem<VPL, PCAP, QPL>*>(smem_raw);
  WarpSmem<VPL, PCAP, QPL>& S = Sw[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  if (lane == 0) S.ct = WarpCounters{};
  __syncwarp();
  long long empties = 0, overflows = 0;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&P.work[0], 1);
    item = __shfl_sync(FULL, item, 0);
    const int si = P.cell_begin + item;
    if (si >= P.cell_end) break;
    const int orig = P.perm[si];
    int* row = P.scratch + (size_t)orig * P.stride;
    int reason = 0;
    // the ambiguous-sign count before the cell, kept in shared memory (not
    // a register live across the whole build)
    if (lane == 0) S.amb_mark = S.ct.fp64amb;
    const bool built = build_cell<VPL, PCAP, QPL, GEN>(P, S, si, row, empties, reason);
    __syncwarp();
    if (lane == 0 && S.ct.fp64amb != S.amb_mark) record_ambiguous(P.st, P.amb_list, P.amb_cap, orig);
    if (!built) {
      overflows++;
      if (P.tape && lane == 0) *reinterpret_cast<int4*>(P.tape + (size_t)si * kTapeStride) = make_int4(-1, 0, 0, 0);
      if (lane == 0) atomicAdd((unsigned long long*)&P.st->ovf_reason[reason], 1ull);
      if (lane == 0) {
        int slot = atomicAdd(&P.st->ovf_count, 1);
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
  __syncwarp();
  flush_warp_counters(P, S.ct, lane, empties, overflows);
}

// ---------------------------------------------------------------- large cells

// Cone test of BVH children in the large-cell traversal: polytopes of at
// most kConeExactMax slots take the exact support over their vertices, those
// above kConeBoxMin the chunk boxes, those in between skip the test. It pays
// for cells with few faces that reach far (the edge of a cluster facing empty
// space: 4x on the paper's clustered sets) and for the largest power cells
// (with helping warps, -17% on power1M), and costs about 4% on the batched
// set, whose mid-sized large cells it rarely prunes.
constexpr int kConeExactMax = 128;
constexpr int kConeBoxMin = 512;

// Filter the staged candidate planes against the polytope; clip by those
// that may cut, nearest plane first. Returns CLIP_EMPTY / CLIP_OVERFLOW, or
// CLIP_NONE (c.dirty set if the polytope changed).
__device__ int big_flush(BigCell& c, const BigArena& A, const float4* __restrict__ sites, Counters& ct,
                         bool counters) {
  const unsigned lane = lane_id();
  const int k = c.nst;
  if (k == 0) return CLIP_NONE;
  c.nst = 0;
  const uint32_t cm = big_filter(c, A, k, ct, counters);
  bool keep = (int)lane < k && ((cm >> lane) & 1u);
  const float dkey = keep ? A.hord[lane] : INFINITY;
  uint32_t km = __ballot_sync(FULL, keep);
  while (km) {
    const uint32_t key = keep ? f2o(dkey) : 0xffffffffu;
    const uint32_t mn = __reduce_min_sync(FULL, key);
    const int src = __ffs(__ballot_sync(FULL, keep && key == mn)) - 1;
    const float4 h = A.hs[src];
    PlaneT<float> Hb;
    Hb.nx = h.x;
    Hb.ny = h.y;
    Hb.nz = h.z;
    Hb.b = h.w;
    Hb.e = A.hse[src];
    const int hj = A.hid[src];
    if ((int)lane == src) keep = false;
    km &= ~(1u << src);
    const int rc = big_clip(c, A, Hb, hj, sites, ct, counters, true);
    if (rc == CLIP_EMPTY || rc == CLIP_OVERFLOW) return rc;
    if (rc == CLIP_DONE) {
      c.dirty = true;
      if (counters) ct.clips++;
    }
  }
  __syncwarp();
  return CLIP_NONE;
}

template <bool GEN>
__device__ int big_leaf(BigCell& c, const BigArena& A, int ref, int si, int orig_i, const CellBuffers& P,
                        Counters& ct, int skip0, int skip1) {
  const unsigned lane = lane_id();
  const Knobs<GEN> K(P.cfg);
  const bool counters = K.counters;
  int first = leaf_first(ref), cnt = leaf_count(ref);
  int j = first + (int)lane;
  bool act = (int)lane < cnt && j != si && (j < skip0 || j >= skip1);
  if (act) act = P.loser[j] == 0;
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  if (act) q = P.sites[j];
  PlaneT<float> H;
  H.nx = H.ny = H.nz = H.b = H.e = 0.0f;
  bool keep = false, dup = false;
  float dkey = INFINITY;
  if (act) {
    float nx = q.x - c.me.x, ny = q.y - c.me.y, nz = q.z - c.me.z;
    float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    dup = nx == 0.0f && ny == 0.0f && nz == 0.0f;
    if (!dup) {
      float beta = 0.5f * (nn + (c.me.w - q.w));
      keep = candidate_test(nx, ny, nz, nn, beta, c.me.w, q.w, c.alo, c.ahi, c.sc, c.srad, K.cull);
      if (keep) {
        H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
        dkey = H.b;
      }
    }
  }
  if (__any_sync(FULL, dup)) {
    bool beats = dup && (q.w > c.me.w || (q.w == c.me.w && P.perm[j] < orig_i));
    if (__any_sync(FULL, beats)) return CLIP_EMPTY;
  }
  uint32_t km = __ballot_sync(FULL, keep);
  if (counters) ct.cand += __popc(km);
  if (!km) return CLIP_NONE;
  // stage the survivors; the staged planes of several leaves are filtered
  // together (a bound computed before their clips is only looser)
  if (c.nst + __popc(km) > 32) {
    const int rc = big_flush(c, A, P.sites, ct, counters);
    if (rc != CLIP_NONE) return rc;
  }
  const int slot = c.nst + __popc(km & lanemask_lt());
  if (keep) {
    A.hs[slot] = make_float4(H.nx, H.ny, H.nz, H.b);
    A.hse[slot] = H.e;
    A.hid[slot] = j;
    A.hord[slot] = dkey;
  }
  c.nst += __popc(km);
  __syncwarp();
  return CLIP_NONE;
}

// Volume and first moment about the vertex mean (same fan tetrahedra as the
// register path), using the pair hash for the edge successors; cells that
// fail the FP32 error estimate are integrated again in FP64, with the FP64
// vertex positions kept in the arena's staging arrays.
__device__ inline void big_volume(const BigCell& c, const BigArena& A, const float4* __restrict__ sites, double& V,
                                  double& ox, double& oy, double& oz, Counters& ct) {
  const uint32_t hmask = big_hash_vertices(c, A);
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    float4 v = A.vp[i];
    sx += v.x;
    sy += v.y;
    sz += v.z;
  }
  const float cx = warp_sumf(sx) / c.nv, cy = warp_sumf(sy) / c.nv, cz = warp_sumf(sz) / c.nv;
  float Vf = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f, Sabs = 0.f, emax = 0.f;
  for (int it = (int)lane_id(); it < 3 * c.nv; it += 32) {
    int t = it / 3, rho = it % 3;
    uint32_t q = bpair(A.vt[t], rho);
    uint32_t fy = q >> 16;
    int u = hash_find(A, brev(q), hmask);
    if (u < 0) continue;
    float4 pf = A.pl[fy];
    float hgt = fmaf(pf.x, cx, fmaf(pf.y, cy, fmaf(pf.z, cz, -pf.w)));
    float gx = -hgt * pf.x, gy = -hgt * pf.y, gz = -hgt * pf.z;
    float4 a = A.vp[t], b = A.vp[u];
    float ax = a.x - cx, ay = a.y - cy, az = a.z - cz;
    float bx = b.x - cx, by = b.y - cy, bz = b.z - cz;
    float det = gx * (ay * bz - az * by) + gy * (az * bx - ax * bz) + gz * (ax * by - ay * bx);
    Vf += det;
    Mx += det * (gx + ax + bx);
    My += det * (gy + ay + by);
    Mz += det * (gz + az + bz);
    float e1x = ax - gx, e1y = ay - gy, e1z = az - gz, e2x = bx - gx, e2y = by - gy, e2z = bz - gz;
    float crx = e1y * e2z - e1z * e2y, cry = e1z * e2x - e1x * e2z, crz = e1x * e2y - e1y * e2x;
    Sabs += sqrtf(crx * crx + cry * cry + crz * crz);
    emax = fmaxf(emax, a.w);
  }
  Vf = warp_sumf(Vf) * (1.0f / 6.0f);
  Mx = warp_sumf(Mx) * (1.0f / 24.0f);
  My = warp_sumf(My) * (1.0f / 24.0f);
  Mz = warp_sumf(Mz) * (1.0f / 24.0f);
  Sabs = warp_sumf(Sabs) * 0.5f;
  emax = warp_maxf(emax);
  float L = 0.f;
#pragma unroll
  for (int k = 0; k < 3; k++) L += fmaxf(c.alo[k] * c.alo[k], c.ahi[k] * c.ahi[k]);
  L = sqrtf(L);
  ox = cx;
  oy = cy;
  oz = cz;
  V = Vf;
  if (!c.fp64 || !volume_needs_fp64(Vf, L, Sabs, emax)) {
    if (Vf > 0.f) {
      ox += Mx / Vf;
      oy += My / Vf;
      oz += Mz / Vf;
    }
    return;
  }
  ct.refvol++;
  // FP64 vertex positions: x, y in nvp (as two doubles), z in otri
  double2* p2 = reinterpret_cast<double2*>(A.nvp);
  double* pz = reinterpret_cast<double*>(A.otri);
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    uint64_t T = A.vt[i];
    double x, y, z;
    vertex64(bfield(T, 0), bfield(T, 1), bfield(T, 2), A.pid, c.me, c.lo, c.hi, sites, x, y, z);
    p2[i] = make_double2(x, y);
    pz[i] = z;
  }
  __syncwarp();
  double Vd = 0.0, Mxd = 0.0, Myd = 0.0, Mzd = 0.0;
  const double dcx = cx, dcy = cy, dcz = cz;
  for (int it = (int)lane_id(); it < 3 * c.nv; it += 32) {
    int t = it / 3, rho = it % 3;
    uint32_t q = bpair(A.vt[t], rho);
    uint32_t fy = q >> 16;
    int u = hash_find(A, brev(q), hmask);
    if (u < 0) continue;
    PlaneT<double> pf = plane64(A.pid[fy], c.me, c.lo, c.hi, sites);
    double hgt = pf.nx * dcx + pf.ny * dcy + pf.nz * dcz - pf.b;
    double gx = -hgt * pf.nx, gy = -hgt * pf.ny, gz = -hgt * pf.nz;
    double2 a2 = p2[t], b2 = p2[u];
    double ax = a2.x - dcx, ay = a2.y - dcy, az = pz[t] - dcz;
    double bx = b2.x - dcx, by = b2.y - dcy, bz = pz[u] - dcz;
    double det = gx * (ay * bz - az * by) + gy * (az * bx - ax * bz) + gz * (ax * by - ay * bx);
    Vd += det;
    Mxd += det * (gx + ax + bx);
    Myd += det * (gy + ay + by);
    Mzd += det * (gz + az + bz);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Vd += __shfl_xor_sync(FULL, Vd, o);
    Mxd += __shfl_xor_sync(FULL, Mxd, o);
    Myd += __shfl_xor_sync(FULL, Myd, o);
    Mzd += __shfl_xor_sync(FULL, Mzd, o);
  }
  V = Vd / 6.0;
  if (V > 0.0) {
    ox += Mxd / 24.0 / V;
    oy += Myd / 24.0 / V;
    oz += Mzd / 24.0 / V;
  }
  __syncwarp();
}

// Returns false if the cell overflowed even the large capacity.
// The finished (compacted) polytope of a large cell on the large-cell tape,
// and the site's tape header pointing at it; a cell that does not fit keeps
// the header -1 (the adjoint re-clips it).
__device__ inline void big_tape_write(const BigCell& c, const BigArena& A, const CellBuffers& P, int si) {
  const unsigned lane = lane_id();
  const long long bytes = big_tape_bytes(c.nv, c.npl);
  unsigned long long off = 0;
  if (lane == 0) off = atomicAdd((unsigned long long*)&P.st->btape_used, (unsigned long long)bytes);
  off = __shfl_sync(FULL, off, 0);
  if ((long long)off + bytes > P.btape_cap) return;
  char* rec = P.btape + off;
  float4* vp = reinterpret_cast<float4*>(rec + 16);
  uint64_t* vt = reinterpret_cast<uint64_t*>(rec + 16 + 16 * (size_t)c.nv);
  int* pid = reinterpret_cast<int*>(rec + 16 + 24 * (size_t)c.nv);
  for (int i = (int)lane; i < c.nv; i += 32) {
    vp[i] = A.vp[i];
    vt[i] = A.vt[i];
  }
  for (int p = (int)lane; p < c.npl; p += 32) pid[p] = A.pid[p];
  if (lane == 0) {
    atomicAdd((unsigned long long*)&P.st->btape_records, 1ull);
    *reinterpret_cast<int4*>(rec) = make_int4(c.nv, c.npl, 0, 0);
    *reinterpret_cast<int4*>(P.tape + (size_t)si * kTapeStride) =
        make_int4(-2, c.npl, (int)(unsigned)(off & 0xffffffffull), (int)(unsigned)(off >> 32));
  }
  __syncwarp();
}

template <bool GEN>
__device__ bool big_build_cell(const CellBuffers& P, const BigArena& A, int si, Counters& ct, long long& empties) {
  const unsigned lane = lane_id(), lt = lanemask_lt();
  const Knobs<GEN> K(P.cfg);
  const bool counters = K.counters;
  BigCell c;
  c.me = P.sites[si];
  c.fp64 = GEN ? P.cfg.precision == 0 : true;
  const int orig_i = P.perm[si];
  const int set = P.nsets > 1 ? (int)(P.keys[si] >> P.set_shift) : 0;
  const SetInfo& SI = P.sets[set];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.lo[k] = SI.lo[k];
    c.hi[k] = SI.hi[k];
  }
  const int cull = K.cull, trav = K.trav;
  big_init(c, A, cull);
  bool empty = false, overflow = false;
  int skip0 = 0, skip1 = 0;
  if (P.cfg.warm_start) {
    const int lo = SI.first, hi = SI.first + SI.count;
    skip0 = max(lo, min(si - 16, hi - 32));
    skip1 = min(hi, skip0 + 32);
    int rc = big_leaf<GEN>(c, A, make_leaf_ref(skip0, skip1 - skip0), si, orig_i, P, ct, 0, 0);
    if (rc == CLIP_NONE) rc = big_flush(c, A, P.sites, ct, counters);
    if (rc == CLIP_EMPTY) empty = true;
    if (rc == CLIP_OVERFLOW) return false;
    if (c.dirty) {
      big_aabb(c, A, cull);
      c.dirty = false;
    }
  }
  int cur = SI.root;
  bool have = !empty;
  while (!empty) {
    if (have) {
      if (ref_is_leaf(cur)) {
        int rc = big_leaf<GEN>(c, A, cur, si, orig_i, P, ct, skip0, skip1);
        if (rc == CLIP_EMPTY) {
          empty = true;
          break;
        }
        if (rc == CLIP_OVERFLOW) {
          overflow = true;
          break;
        }
        if (c.dirty) {
          big_aabb(c, A, cull);
          c.dirty = false;
        }
        have = false;
      } else {
        const float4* nd = P.nodes + 4 * (size_t)cur;
        float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < 4) rec = __ldg(nd + lane);
        float4 hi;
        hi.x = __shfl_down_sync(FULL, rec.x, 1);
        hi.y = __shfl_down_sync(FULL, rec.y, 1);
        hi.z = __shfl_down_sync(FULL, rec.z, 1);
        hi.w = __shfl_down_sync(FULL, rec.w, 1);
        float lb = 0.f, key = 0.f;
        int occ = 0;
        bool keep = false;
        if (lane == 0 || lane == 2) keep = node_test(rec, hi, c.me, A.rtab, cull, lb, occ, key);
        int myref = __float_as_int(hi.w);
        bool k0 = __shfl_sync(FULL, keep, 0), k1 = __shfl_sync(FULL, keep, 2);
        float key0 = __shfl_sync(FULL, key, 0), key1 = __shfl_sync(FULL, key, 2);
        int r0 = __shfl_sync(FULL, myref, 0), r1 = __shfl_sync(FULL, myref, 2);
        if (counters) ct.nodes += 2;
        // cone bound of each surviving child: the cell's support in the cone
        // axis, exact over the vertices of a small polytope (dead slots are
        // NaN: ignored), over the chunk boxes of a large one
        if ((k0 || k1) && cull == 0 && (c.nv <= kConeExactMax || c.nv > kConeBoxMin)) {
          const float rmax = sqrtf(c.sc[0] * c.sc[0] + c.sc[1] * c.sc[1] + c.sc[2] * c.sc[2]) + c.srad;
#pragma unroll
          for (int ch = 0; ch < 2; ch++) {
            const bool kc = ch == 0 ? k0 : k1;
            if (!kc) continue;
            const int src = 2 * ch;
            float4 blo, bhi;
            blo.x = __shfl_sync(FULL, rec.x, src);
            blo.y = __shfl_sync(FULL, rec.y, src);
            blo.z = __shfl_sync(FULL, rec.z, src);
            bhi.x = __shfl_sync(FULL, hi.x, src);
            bhi.y = __shfl_sync(FULL, hi.y, src);
            bhi.z = __shfl_sync(FULL, hi.z, src);
            const float lbc = __shfl_sync(FULL, lb, src);
            Cone k;
            if (!node_cone(blo, bhi, c.me, k)) continue;
            float h = -INFINITY;
            if (c.nv <= kConeExactMax) {
              for (int i = (int)lane; i < c.nv; i += 32) {
                const float4 v = A.vp[i];
                h = fmaxf(h, fmaf(k.ux, v.x, fmaf(k.uy, v.y, k.uz * v.z)));
              }
            } else {
              const int nch = (c.nv + 31) >> 5;
              for (int q = (int)lane; q < nch; q += 32) {
                const float4 qlo = A.cb[2 * q], qhi = A.cb[2 * q + 1];
                if (!(qlo.x <= qhi.x)) continue;  // every slot of the chunk dead
                const float sx = k.ux >= 0.0f ? qhi.x : qlo.x, sy = k.uy >= 0.0f ? qhi.y : qlo.y,
                            sz = k.uz >= 0.0f ? qhi.z : qlo.z;
                h = fmaxf(h, fmaf(k.ux, sx, fmaf(k.uy, sy, k.uz * sz)));
              }
            }
            h = warp_maxf(h);
            if (cone_culls(lbc, h, c.em, rmax, k)) {
              if (ch == 0)
                k0 = false;
              else
                k1 = false;
            }
          }
        }
        if (k0 && k1) {
          bool near0 = key0 <= key1;  // nearer child first (both traversals)
          int fsrc = near0 ? 2 : 0;
          float flb = __shfl_sync(FULL, lb, fsrc);
          int focc = __shfl_sync(FULL, occ, fsrc);
          cur = near0 ? r0 : r1;
          if (!big_push(c, A, flb, near0 ? key1 : key0, trav, near0 ? r1 : r0, focc)) {
            overflow = true;
            break;
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
    if (!big_pop(c, A, cull, cur)) break;
    have = true;
  }
  if (!empty && !overflow) {
    const int rc = big_flush(c, A, P.sites, ct, counters);
    if (rc == CLIP_EMPTY) empty = true;
    if (rc == CLIP_OVERFLOW) overflow = true;
    if (c.dirty) {
      big_aabb(c, A, cull);
      c.dirty = false;
    }
  }
  if (overflow) return false;
  if (empty) {
    if (lane == 0) {
      P.counts[orig_i] = 0;
      P.vol[orig_i] = 0.0f;
      P.cen[3 * (size_t)orig_i] = c.me.x;
      P.cen[3 * (size_t)orig_i + 1] = c.me.y;
      P.cen[3 * (size_t)orig_i + 2] = c.me.z;
    }
    empties++;
    return true;
  }
  big_compact(c, A);
  // neighbours: site planes that carry a face, sorted, into the pool
  big_mark_planes(c, A);
  int* list = reinterpret_cast<int*>(A.otri);
  int cnt = 0;
  for (int base = 0; base < c.npl; base += 32) {
    int p = base + (int)lane;
    bool isn = p < c.npl && A.flag[p] != 0 && A.pid[p] >= 0;
    uint32_t mk = __ballot_sync(FULL, isn);
    if (isn) list[cnt + __popc(mk & lt)] = P.perm[A.pid[p]] - SI.first;
    cnt += __popc(mk);
  }
  __syncwarp();
  if (P.btape && P.tape) big_tape_write(c, A, P, si);
  long long off = 0;
  if (cnt <= P.stride) {
    // short list: the cell's regular row
    int* row = P.scratch + (size_t)orig_i * P.stride;
    for (int t = (int)lane; t < cnt; t += 32) {
      int v = list[t];
      int rank = 0;
      for (int u = 0; u < cnt; u++) rank += list[u] < v;
      row[rank] = v;
    }
    if (lane == 0) P.counts[orig_i] = cnt;
  } else if (lane == 0) {
    off = atomicAdd((unsigned long long*)&P.st->pool_used, (unsigned long long)cnt);
  }
  off = __shfl_sync(FULL, off, 0);
  if (cnt <= P.stride) {
  } else if (off + cnt > P.pool_cap) {
    if (lane == 0) {
      P.counts[orig_i] = 0;
      set_error(P.st, VD_ERR_CELL_OVERFLOW);
    }
  } else {
    for (int t = (int)lane; t < cnt; t += 32) {
      int v = list[t];
      int rank = 0;
      for (int u = 0; u < cnt; u++) rank += list[u] < v;
      P.pool[off + rank] = v;
    }
    if (lane == 0) {
      P.counts[orig_i] = cnt;
      P.ovf_slot[orig_i] = (int)off;
    }
  }
  double V, ox, oy, oz;
  big_volume(c, A, P.sites, V, ox, oy, oz, ct);
  if (lane == 0) {
    P.vol[orig_i] = (float)V;
    P.cen[3 * (size_t)orig_i] = (float)((double)c.me.x + ox);
    P.cen[3 * (size_t)orig_i + 1] = (float)((double)c.me.y + oy);
    P.cen[3 * (size_t)orig_i + 2] = (float)((double)c.me.z + oz);
  }
  __syncwarp();
  return true;
}

template <bool GEN>
__global__ void __launch_bounds__(32 * kBigWarpsPerBlock, kBigBlocksPerSm) big_cells_kernel(CellBuffers P) {
  const unsigned lane = lane_id();
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  BigArena A = big_arena(P.arena, slot);
  extern __shared__ __align__(16) char big_smem[];
  A.hb = reinterpret_cast<HelpBoard*>(big_smem + kBigSmemPerWarp * kBigWarpsPerBlock);
  A.err = &P.st->error;
  A.stall = P.stall;
  if (threadIdx.x < kBigWarpsPerBlock) {
    A.hb->req[threadIdx.x].seq = 0;
    A.hb->req[threadIdx.x].next = 0;
  }
  if (threadIdx.x == 0) A.hb->live = (int)(blockDim.x >> 5);
  __syncthreads();
  Counters ct = {};
  long long empties = 0, failed = 0;
  const int total = min(P.st->ovf_count, P.ovf_cap);
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&P.work[1], 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    const int si = P.ovf_list[item];
    const long long amb0 = ct.fp64amb;
    const bool built = big_build_cell<GEN>(P, A, si, ct, empties);
    if (__any_sync(FULL, ct.fp64amb != amb0) && lane == 0) record_ambiguous(P.st, P.amb_list, P.amb_cap, P.perm[si]);
    if (!built) {
      failed++;
      if (lane == 0) {
        const int orig = P.perm[si];
        P.counts[orig] = 0;
        P.vol[orig] = __int_as_float(0x7fc00000);
        set_error(P.st, VD_ERR_CELL_OVERFLOW);
      }
    }
  }
  {
    long long tested = 0;
    big_help(A, tested);
    if (GEN && P.cfg.counters) ct.vtests += tested;
  }
  flush_counters(P, ct, lane, empties, 0, failed);
}

template <int VPL, int PCAP, int QPL>
static cudaError_t launch_variant(const CellBuffers& c, int num_sms, cudaStream_t s) {
  int wpb = c.cfg.warps_per_block;
  size_t smem = sizeof(WarpSmem<VPL, PCAP, QPL>) * (size_t)wpb;
  const bool generic = c.cfg.cull_mode != 0 || c.cfg.traversal != 0 || c.cfg.counters != 0 || c.cfg.precision != 0;
  auto kern = generic ? cells_kernel<VPL, PCAP, QPL, true> : cells_kernel<VPL, PCAP, QPL, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = c.cfg.blocks_per_sm;
  if (per_sm <= 0) {
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * wpb, smem);
    if (err != cudaSuccess) return err;
    per_sm = occ > 0 ? occ : 1;
  }
  kern<<<num_sms * per_sm, 32 * wpb, smem, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cells(const CellBuffers& c, int num_sms, cudaStream_t s, const std::function<void()>& between) {
  cudaError_t err;
  const vd_config& g = c.cfg;
  const int q = g.queue_per_lane;
  if (g.cell_mode == 1) {
    err = launch_cells_thread(c, num_sms, s);
  } else if (g.verts_per_lane >= 4) {
    err = q >= 8   ? launch_variant<4, 128, 8>(c, num_sms, s)
          : q >= 4 ? launch_variant<4, 128, 4>(c, num_sms, s)
          : q >= 2 ? launch_variant<4, 128, 2>(c, num_sms, s)
                   : launch_variant<4, 128, 1>(c, num_sms, s);
  } else {
    err = q >= 8   ? launch_variant<2, 64, 8>(c, num_sms, s)
          : q >= 4 ? launch_variant<2, 64, 4>(c, num_sms, s)
          : q >= 2 ? launch_variant<2, 64, 2>(c, num_sms, s)
                   : launch_variant<2, 64, 1>(c, num_sms, s);
  }
  if (err != cudaSuccess) return err;
  between();
  // cells that overflowed the register-resident capacity
  const size_t big_smem = kBigSmemPerWarp * kBigWarpsPerBlock + sizeof(HelpBoard);
  const vd_config& gc = c.cfg;
  auto big = (gc.cull_mode != 0 || gc.traversal != 0 || gc.counters != 0 || gc.precision != 0) ? big_cells_kernel<true>
                                                                                                : big_cells_kernel<false>;
  err = cudaFuncSetAttribute(big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
  if (err != cudaSuccess) return err;
  big<<<num_sms * kBigBlocksPerSm, 32 * kBigWarpsPerBlock, big_smem, s>>>(c);
  return cudaGetLastError();
}

}  // namespace vd
