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

#include "vd_clip.cuh"

namespace vd {

// Candidate pre-test of Sec. 4.2.1: the plane n.x <= beta can cut the cell
// only if it cuts the cell's AABB, i.e. n.c_o > beta for the AABB corner c_o
// of n's octant (the exact support of the box in direction n; the paper's
// per-octant corner distance |c_o| bounds it from above).
__device__ __forceinline__ bool candidate_test(float nx, float ny, float nz, float nn, float beta, float wi,
                                               float wj, const float* alo, const float* ahi, int cull_mode) {
  if (cull_mode == 2) return true;
  float n[3] = {nx, ny, nz};
  float pad = 0.5f * (nn + fabsf(wi) + fabsf(wj));
  if (cull_mode == 1) {
    float R = sqrtf(dir_radius2(0, alo, ahi, 1));
    float len = sqrtf(nn);
    pad = kCullPad * (pad + len * R);
    return len * R * (1.0f + kCullPad) > beta - pad;
  }
  float sup = 0.0f, mag = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float t = n[k] > 0.0f ? n[k] * ahi[k] : (n[k] < 0.0f ? n[k] * alo[k] : 0.0f);
    sup += t;
    mag += fabsf(t);
  }
  return sup > beta - kCullPad * (pad + mag);
}

// Process the sites of one leaf: pre-cull all of them in parallel, then
// clip with the survivors in ascending power distance d_ij (Eq. 2).
template <int VPL, int PCAP, int QPL>
__device__ int process_leaf(Cell<VPL, PCAP, QPL>& c, WarpSmem<VPL, PCAP>& S, int ref, int si, int orig_i,
                            const CellBuffers& P, Counters& ct) {
  const unsigned lane = lane_id();
  const bool counters = P.cfg.counters != 0;
  int first = leaf_first(ref), cnt = leaf_count(ref);
  int j = first + (int)lane;
  bool act = (int)lane < cnt && j != si;
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
      keep = candidate_test(nx, ny, nz, nn, beta, c.me.w, q.w, c.alo, c.ahi, P.cfg.cull_mode);
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
  if (counters) ct.cand += __popc(km);
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
    if ((int)lane == src) keep = false;
    km &= ~(1u << src);
    int rc = clip_cell(c, S, Hb, first + src, P.sites, ct, counters);
    if (rc == CLIP_EMPTY || rc == CLIP_OVERFLOW) return rc;
    if (rc == CLIP_DONE) {
      c.dirty = true;
      if (counters) ct.clips++;
    }
  }
  return CLIP_NONE;
}

// Build one cell and write its outputs. Returns false on overflow.
template <int VPL, int PCAP, int QPL>
__device__ bool build_cell(const CellBuffers& P, WarpSmem<VPL, PCAP>& S, int si, int* row, Counters& ct,
                           long long& empties) {
  using C = Cell<VPL, PCAP, QPL>;
  constexpr int NPW = C::NPW;
  const unsigned lane = lane_id(), lt = lanemask_lt();
  const bool counters = P.cfg.counters != 0;
  C c;
  c.me = P.sites[si];
  const int orig_i = P.perm[si];
  const int set = P.nsets > 1 ? (int)(P.keys[si] >> P.set_shift) : 0;
  const SetInfo& SI = P.sets[set];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.lo[k] = SI.lo[k];
    c.hi[k] = SI.hi[k];
  }
  init_cell(c, S);

  // ---- best-first traversal (Alg. 1)
  bool empty = false, overflow = false;
  int cur = SI.root;
  bool have = true;
  const int cull = P.cfg.cull_mode, trav = P.cfg.traversal;
  while (true) {
    if (have) {
      if (ref_is_leaf(cur)) {
        int rc = process_leaf(c, S, cur, si, orig_i, P, ct);
        if (rc == CLIP_EMPTY) {
          empty = true;
          break;
        }
        if (rc == CLIP_OVERFLOW) {
          overflow = true;
          break;
        }
        if (c.dirty) {
          recompute_aabb(c);
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
        if (lane == 0 || lane == 2) keep = node_test(rec, hi, c.me, c.alo, c.ahi, cull, lb, occ, key);
        int myref = __float_as_int(hi.w);
        bool k0 = __shfl_sync(FULL, keep, 0), k1 = __shfl_sync(FULL, keep, 2);
        float key0 = __shfl_sync(FULL, key, 0), key1 = __shfl_sync(FULL, key, 2);
        int r0 = __shfl_sync(FULL, myref, 0), r1 = __shfl_sync(FULL, myref, 2);
        if (counters) ct.nodes += 2;
        if (k0 && k1) {
          bool near0 = trav == 1 ? true : key0 <= key1;
          int fsrc = near0 ? 2 : 0;
          float flb = __shfl_sync(FULL, lb, fsrc);
          int focc = __shfl_sync(FULL, occ, fsrc);
          cur = near0 ? r0 : r1;
          if (!queue_push(c, flb, near0 ? r1 : r0, focc)) {
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
    if (!queue_pop(c, cull, trav, cur)) break;
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
  // neighbours: site planes that carry a face
  int nvals = 0;
  const int setfirst = SI.first;
#pragma unroll
  for (int w = 0; w < NPW; w++) {
    int f = 32 * w + (int)lane;
    bool isn = ((alive[w] >> lane) & 1u) && S.pid[f] >= 0;
    uint32_t mk = __ballot_sync(FULL, isn);
    if (isn) S.otri[nvals + __popc(mk & lt)] = (uint32_t)(P.perm[S.pid[f]] - setfirst);
    nvals += __popc(mk);
  }
  __syncwarp();
  for (int t = (int)lane; t < nvals; t += 32) {
    int v = (int)S.otri[t];
    int rank = 0;
    for (int u = 0; u < nvals; u++) rank += (int)S.otri[u] < v;
    row[rank] = v;
  }
  // volume and first moment: tetrahedra (c, g_f, v, w) for every directed
  // edge v -> w of face f (w = the other end of the edge), g_f = the foot of
  // c on plane f; c = vertex mean
  float cx = sx / nv, cy = sy / nv, cz = sz / nv;
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
  }
  V = warp_sumf(V) * (1.0f / 6.0f);
  Mx = warp_sumf(Mx) * (1.0f / 24.0f);
  My = warp_sumf(My) * (1.0f / 24.0f);
  Mz = warp_sumf(Mz) * (1.0f / 24.0f);
  if (lane == 0) {
    P.counts[orig_i] = nvals;
    vol[orig_i] = V;
    float ox = cx, oy = cy, oz = cz;
    if (V > 0.0f) {
      ox += Mx / V;
      oy += My / V;
      oz += Mz / V;
    }
    cen[3 * (size_t)orig_i] = c.me.x + ox;
    cen[3 * (size_t)orig_i + 1] = c.me.y + oy;
    cen[3 * (size_t)orig_i + 2] = c.me.z + oz;
  }
  __syncwarp();
  return true;
}

template <int VPL, int PCAP, int QPL, bool BIG>
__global__ void cells_kernel(CellBuffers P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<VPL, PCAP>* Sw = reinterpret_cast<WarpSmem<VPL, PCAP>*>(smem_raw);
  WarpSmem<VPL, PCAP>& S = Sw[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  Counters ct = {0, 0, 0, 0, 0, 0, 0};
  long long empties = 0, overflows = 0, failed = 0;
  const int total = BIG ? min(P.st->ovf_count, P.ovf_cap) : P.n;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&P.work[BIG ? 1 : 0], 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    int si = BIG ? P.ovf_list[item] : item;
    int orig = P.perm[si];
    int* row = BIG ? P.scratch_big + (size_t)item * P.stride_big : P.scratch + (size_t)orig * P.stride;
    bool ok = build_cell<VPL, PCAP, QPL>(P, S, si, row, ct, empties);
    if (!ok) {
      if (BIG) {
        failed++;
        if (lane == 0) {
          P.counts[orig] = 0;
          P.vol[orig] = __int_as_float(0x7fc00000);
          set_error(P.st, VD_ERR_CELL_OVERFLOW);
        }
      } else {
        overflows++;
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
    } else if (BIG && lane == 0) {
      P.ovf_slot[orig] = item;
    }
  }
  if (lane == 0) {
    if (empties) atomicAdd((unsigned long long*)&P.st->empty_cells, (unsigned long long)empties);
    if (overflows) atomicAdd((unsigned long long*)&P.st->overflow_cells, (unsigned long long)overflows);
    if (failed) atomicAdd((unsigned long long*)&P.st->failed_cells, (unsigned long long)failed);
  }
  // per-lane counters (FP64 re-evaluations happen on individual lanes)
  long long f64 = ct.fp64, f64a = ct.fp64amb;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f64 += __shfl_xor_sync(FULL, f64, o);
    f64a += __shfl_xor_sync(FULL, f64a, o);
  }
  if (lane == 0) {
    if (f64) atomicAdd((unsigned long long*)&P.st->fp64_fallbacks, (unsigned long long)f64);
    if (f64a) atomicAdd((unsigned long long*)&P.st->fp64_ambiguous, (unsigned long long)f64a);
    if (P.cfg.counters) {
      atomicAdd((unsigned long long*)&P.st->candidates, (unsigned long long)ct.cand);
      atomicAdd((unsigned long long*)&P.st->clips, (unsigned long long)ct.clips);
      atomicAdd((unsigned long long*)&P.st->nodes, (unsigned long long)ct.nodes);
      atomicAdd((unsigned long long*)&P.st->vertex_tests, (unsigned long long)ct.vtests);
      atomicAdd((unsigned long long*)&P.st->new_vertices, (unsigned long long)ct.newv);
    }
  }
}

template <int VPL, int PCAP, int QPL, bool BIG>
static cudaError_t launch_variant(const CellBuffers& c, int num_sms, int grid_override, cudaStream_t s) {
  int wpb = c.cfg.warps_per_block;
  if (BIG) wpb = 4;
  size_t smem = sizeof(WarpSmem<VPL, PCAP>) * (size_t)wpb;
  auto kern = cells_kernel<VPL, PCAP, QPL, BIG>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = c.cfg.blocks_per_sm;
  if (per_sm <= 0 || BIG) {
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * wpb, smem);
    if (err != cudaSuccess) return err;
    per_sm = occ > 0 ? occ : 1;
  }
  int grid = grid_override > 0 ? grid_override : num_sms * per_sm;
  kern<<<grid, 32 * wpb, smem, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cells(const CellBuffers& c, int num_sms, cudaStream_t s, const std::function<void()>& between) {
  cudaError_t err;
  const vd_config& g = c.cfg;
  if (g.verts_per_lane >= 4) {
    err = g.queue_per_lane >= 2 ? launch_variant<4, 64, 2, false>(c, num_sms, 0, s)
                                : launch_variant<4, 64, 1, false>(c, num_sms, 0, s);
  } else {
    err = g.queue_per_lane >= 2 ? launch_variant<2, 64, 2, false>(c, num_sms, 0, s)
                                : launch_variant<2, 64, 1, false>(c, num_sms, 0, s);
  }
  if (err != cudaSuccess) return err;
  between();
  // cells that overflowed the register-resident capacity: large-capacity
  // pass (256 vertices, 192 planes, 256 queue entries)
  return launch_variant<8, 192, 8, true>(c, num_sms, num_sms * 2, s);
}

}  // namespace vd
