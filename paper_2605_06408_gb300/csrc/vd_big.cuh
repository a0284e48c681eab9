// vd_big.cuh -- the large-cell path.
//
// Cells whose polytope outgrows the register-resident capacity (sliver cells
// of anisotropic clusters, cells of large-weight sites with thousands of
// faces) are rebuilt by this path: the same traversal, culling and clipping
// steps, with the polytope, the plane list, the best-first queue and a pair
// hash held in a per-warp arena of global memory, as the paper keeps its
// per-thread state in global memory (App. A.3). Planes are compacted when
// the plane array passes 85% occupancy (App. A.4). Plane indices are 16-bit,
// vertex triplets 64-bit (a | b<<16 | c<<32, bit 63 = "outside" mark).
#pragma once

#include "vd_clip.cuh"

namespace vd {

constexpr int kBigV = 16384;   // vertices per cell
constexpr int kBigP = 8192;    // planes per cell
constexpr int kBigQ = 8192;    // queue entries
constexpr int kBigH = 65536;   // pair-hash slots (power of two)
constexpr int kBigGc = (kBigP * 85) / 100;
constexpr uint64_t kBigOut = 1ull << 63;
constexpr uint64_t kTriMask = 0x0000ffffffffffffull;
constexpr uint32_t kHashEmpty = 0xffffffffu;

struct BigArena {
  float4* pl;
  float* pe;
  int* pid;
  int* flag;
  float4* vp;
  uint64_t* vt;
  uint64_t* otri;
  float4* nvp;
  uint64_t* nvt;
  float* qlb;
  int* qref;
  int* qocc;
  uint32_t* hkey;
  int* hval;
  float* acc;
  float* rtab;  // [64] cell radius per occupied-octant mask
};

__host__ __device__ inline size_t big_arena_bytes() {
  size_t b = 64 * 4;
  b += (size_t)kBigP * (16 + 4 + 4 + 4);
  b += (size_t)kBigV * (16 + 8 + 8 + 16 + 8);
  b += (size_t)kBigQ * 12;
  b += (size_t)kBigH * 8;
  b += (size_t)kBigP * 10 * 4;
  return (b + 255) & ~(size_t)255;
}

__device__ inline BigArena big_arena(char* base, int slot) {
  char* p = base + (size_t)slot * big_arena_bytes();
  BigArena A;
  A.pl = (float4*)p;
  p += (size_t)kBigP * 16;
  A.vp = (float4*)p;
  p += (size_t)kBigV * 16;
  A.nvp = (float4*)p;
  p += (size_t)kBigV * 16;
  A.vt = (uint64_t*)p;
  p += (size_t)kBigV * 8;
  A.otri = (uint64_t*)p;
  p += (size_t)kBigV * 8;
  A.nvt = (uint64_t*)p;
  p += (size_t)kBigV * 8;
  A.pe = (float*)p;
  p += (size_t)kBigP * 4;
  A.pid = (int*)p;
  p += (size_t)kBigP * 4;
  A.flag = (int*)p;
  p += (size_t)kBigP * 4;
  A.qlb = (float*)p;
  p += (size_t)kBigQ * 4;
  A.qref = (int*)p;
  p += (size_t)kBigQ * 4;
  A.qocc = (int*)p;
  p += (size_t)kBigQ * 4;
  A.hkey = (uint32_t*)p;
  p += (size_t)kBigH * 4;
  A.hval = (int*)p;
  p += (size_t)kBigH * 4;
  A.acc = (float*)p;
  p += (size_t)kBigP * 10 * 4;
  A.rtab = (float*)p;
  return A;
}

struct BigCell {
  float4 me;
  float lo[3], hi[3];
  float alo[3], ahi[3];
  float sc[3], srad;
  int nv, npl, qn, seq;
  bool dirty;
};

// ---------------------------------------------------------------- triplets
__device__ __forceinline__ uint64_t btri(uint32_t a, uint32_t b, uint32_t c) {
  return (uint64_t)a | ((uint64_t)b << 16) | ((uint64_t)c << 32);
}
__device__ __forceinline__ uint32_t bfield(uint64_t T, int i) { return (uint32_t)(T >> (16 * i)) & 0xffffu; }
// cyclic pair c of T as x | y << 16
__device__ __forceinline__ uint32_t bpair(uint64_t T, int c) {
  T &= kTriMask;
  uint64_t U = T | (T << 48);
  return (uint32_t)(U >> (16 * c));
}
__device__ __forceinline__ bool bhas(uint64_t T, uint32_t q) {
  return bpair(T, 0) == q || bpair(T, 1) == q || bpair(T, 2) == q;
}
__device__ __forceinline__ uint32_t brev(uint32_t q) { return (q >> 16) | (q << 16); }

// ---------------------------------------------------------------- pair hash
__device__ __forceinline__ uint32_t hash_slot(uint32_t key, uint32_t mask) {
  uint32_t h = key * 2654435761u;
  h ^= h >> 15;
  return h & mask;
}
__device__ __forceinline__ uint32_t hash_size(int entries) {
  uint32_t s = 64;
  while (s < (uint32_t)(2 * entries) && s < (uint32_t)kBigH) s <<= 1;
  return s;
}
__device__ __forceinline__ void hash_clear(const BigArena& A, uint32_t size) {
  for (uint32_t i = lane_id(); i < size; i += 32) A.hkey[i] = kHashEmpty;
  __syncwarp();
}
__device__ __forceinline__ void hash_insert(const BigArena& A, uint32_t key, int val, uint32_t mask) {
  uint32_t s = hash_slot(key, mask);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    uint32_t prev = atomicCAS(&A.hkey[s], kHashEmpty, key);
    if (prev == kHashEmpty || prev == key) {
      A.hval[s] = val;
      return;
    }
    s = (s + 1) & mask;
  }
}
__device__ __forceinline__ int hash_find(const BigArena& A, uint32_t key, uint32_t mask) {
  uint32_t s = hash_slot(key, mask);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    uint32_t k = A.hkey[s];
    if (k == key) return A.hval[s];
    if (k == kHashEmpty) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

// ---------------------------------------------------------------- cell state
__device__ __forceinline__ PlaneT<float> big_plane(const BigArena& A, int k) {
  float4 t = A.pl[k];
  PlaneT<float> P;
  P.nx = t.x;
  P.ny = t.y;
  P.nz = t.z;
  P.b = t.w;
  P.e = A.pe[k];
  return P;
}

__device__ inline void big_aabb(BigCell& c, const BigArena& A, int cull_mode) {
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, em = 0.0f;
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    float4 v = A.vp[i];
    mn[0] = fminf(mn[0], v.x);
    mn[1] = fminf(mn[1], v.y);
    mn[2] = fminf(mn[2], v.z);
    mx[0] = fmaxf(mx[0], v.x);
    mx[1] = fmaxf(mx[1], v.y);
    mx[2] = fmaxf(mx[2], v.z);
    em = fmaxf(em, v.w);
  }
  em = warp_maxf(em);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.alo[k] = warp_minf(mn[k]) - em;
    c.ahi[k] = warp_maxf(mx[k]) + em;
    c.sc[k] = 0.5f * (c.alo[k] + c.ahi[k]);
  }
  float r2 = 0.0f;
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    float4 v = A.vp[i];
    float dx = v.x - c.sc[0], dy = v.y - c.sc[1], dz = v.z - c.sc[2];
    r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
  }
  c.srad = (sqrtf(warp_maxf(r2)) + em) * (1.0f + kCullPad);
  fill_rtab(A.rtab, c.alo, c.ahi, c.sc, c.srad, cull_mode);
}

__device__ inline void big_init(BigCell& c, const BigArena& A, int cull_mode) {
  const unsigned lane = lane_id();
  if (lane < 6) {
    PlaneT<float> B = box_plane<float>((int)lane, c.me.x, c.me.y, c.me.z, c.lo, c.hi);
    A.pl[lane] = make_float4(B.nx, B.ny, B.nz, B.b);
    A.pe[lane] = B.e;
    A.pid[lane] = -1 - (int)lane;
  }
  __syncwarp();
  if (lane < 8) {
    int sx = lane & 1, sy = (lane >> 1) & 1, sz = (lane >> 2) & 1;
    int a = sx, b = 2 + sy, d = 4 + sz;
    if ((sx + sy + sz) & 1) {
      int t = b;
      b = d;
      d = t;
    }
    float x, y, z, e;
    vertex3<float>(big_plane(A, a), big_plane(A, b), big_plane(A, d), x, y, z, e);
    A.vp[lane] = make_float4(x, y, z, e);
    A.vt[lane] = btri(a, b, d);
  }
  c.nv = 8;
  c.npl = 6;
  c.qn = 0;
  c.seq = 0;
  c.dirty = false;
  __syncwarp();
  big_aabb(c, A, cull_mode);
}

// Mark the planes referenced by the vertices in A.flag (1 / 0).
__device__ inline void big_mark_planes(const BigCell& c, const BigArena& A) {
  for (int p = (int)lane_id(); p < c.npl; p += 32) A.flag[p] = 0;
  __syncwarp();
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    uint64_t T = A.vt[i];
#pragma unroll
    for (int f = 0; f < 3; f++) A.flag[bfield(T, f)] = 1;
  }
  __syncwarp();
}

// Plane garbage collection (App. A.4): drop planes no vertex references,
// compact the rest in place and renumber the vertex triplets.
__device__ inline void big_gc(BigCell& c, const BigArena& A) {
  const unsigned lane = lane_id(), lt = lanemask_lt();
  big_mark_planes(c, A);
  int alive = 0;
  for (int base = 0; base < c.npl; base += 32) {
    int p = base + (int)lane;
    bool f = p < c.npl && A.flag[p] != 0;
    uint32_t m = __ballot_sync(FULL, f);
    int dst = alive + __popc(m & lt);
    float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
    float E = 0.f;
    int id = 0;
    if (f) {
      P = A.pl[p];
      E = A.pe[p];
      id = A.pid[p];
    }
    __syncwarp();
    if (f) {
      A.pl[dst] = P;
      A.pe[dst] = E;
      A.pid[dst] = id;
      A.flag[p] = dst;
    }
    alive += __popc(m);
    __syncwarp();
  }
  for (int i = (int)lane; i < c.nv; i += 32) {
    uint64_t T = A.vt[i];
    A.vt[i] = btri(A.flag[bfield(T, 0)], A.flag[bfield(T, 1)], A.flag[bfield(T, 2)]);
  }
  c.npl = alive;
  __syncwarp();
}

static __device__ __noinline__ bool big_resolve64(const BigArena& A, uint64_t tri, int hpid, float4 me, const float* lo,
                                           const float* hi, const float4* __restrict__ sites, long long& amb) {
  PlaneT<double> P0 = plane64(A.pid[bfield(tri, 0)], me, lo, hi, sites);
  PlaneT<double> P1 = plane64(A.pid[bfield(tri, 1)], me, lo, hi, sites);
  PlaneT<double> P2 = plane64(A.pid[bfield(tri, 2)], me, lo, hi, sites);
  double x, y, z, e;
  vertex3<double>(P0, P1, P2, x, y, z, e);
  PlaneT<double> H = plane64(hpid, me, lo, hi, sites);
  double s = side<double>(H, x, y, z);
  if (ambiguous<double>(s, e, H.e)) amb++;
  return s > 0.0;
}

// Clip by plane H of site hpid (App. B), memory-resident form.
static __device__ int big_clip(BigCell& c, const BigArena& A, const PlaneT<float>& H, int hpid,
                        const float4* __restrict__ sites, Counters& ct, bool counters) {
  const unsigned lane = lane_id(), lt = lanemask_lt();
  if (c.npl >= kBigGc) big_gc(c, A);
  if (c.npl >= kBigP) return CLIP_OVERFLOW;
  // read-only first pass (four independent loads per lane in flight): most
  // candidates cut nothing and end here without writes
  {
    bool any = false;
    for (int base = 0; base < c.nv && !any; base += 128) {
      bool o = false;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        int i = base + 32 * u + (int)lane;
        if (i < c.nv) {
          float4 v = A.vp[i];
          float s = side<float>(H, v.x, v.y, v.z);
          bool out = s > 0.0f;
          if (ambiguous<float>(s, v.w, H.e)) out = true;  // settled in FP64 by the marking pass
          o = o || out;
        }
      }
      any = __any_sync(FULL, o);
    }
    if (counters) ct.vtests += c.nv;
    if (!any) return CLIP_NONE;
  }
  // classify; mark outside vertices and list their triplets
  int k = 0;
  for (int base = 0; base < c.nv; base += 32) {
    int i = base + (int)lane;
    bool out = false;
    uint64_t T = 0;
    if (i < c.nv) {
      float4 v = A.vp[i];
      T = A.vt[i];
      float s = side<float>(H, v.x, v.y, v.z);
      out = s > 0.0f;
      if (ambiguous<float>(s, v.w, H.e)) {
        ct.fp64++;
        out = big_resolve64(A, T, hpid, c.me, c.lo, c.hi, sites, ct.fp64amb);
      }
    }
    uint32_t m = __ballot_sync(FULL, out);
    if (out) {
      A.otri[k + __popc(m & lt)] = T;
      A.vt[i] = T | kBigOut;
    }
    k += __popc(m);
  }
  __syncwarp();
  if (k == 0) return CLIP_NONE;
  if (k == c.nv) return CLIP_EMPTY;
  const int h = c.npl++;
  if (lane == 0) {
    A.pl[h] = make_float4(H.nx, H.ny, H.nz, H.b);
    A.pe[h] = H.e;
    A.pid[h] = hpid;
  }
  // hole boundary: directed pairs of outside vertices whose reverse pair
  // belongs to no other outside vertex
  const int E = 3 * k;
  const bool hashed = k > 32;
  uint32_t hmask = 0;
  if (hashed) {
    uint32_t hs = hash_size(E);
    hmask = hs - 1;
    hash_clear(A, hs);
    for (int e = (int)lane; e < E; e += 32) hash_insert(A, bpair(A.otri[e / 3], e % 3), e / 3, hmask);
  }
  __syncwarp();
  int m = 0;
  for (int e0 = 0; e0 < E; e0 += 32) {
    int e = e0 + (int)lane;
    bool isnew = false;
    uint32_t a = 0, b = 0;
    if (e < E) {
      uint32_t q = bpair(A.otri[e / 3], e % 3);
      a = q & 0xffffu;
      b = q >> 16;
      uint32_t rq = brev(q);
      bool interior;
      if (hashed) {
        interior = hash_find(A, rq, hmask) >= 0;
      } else {
        interior = false;
        for (int v = 0; v < k && !interior; v++) interior = bhas(A.otri[v], rq);
      }
      isnew = !interior;
    }
    uint32_t nm = __ballot_sync(FULL, isnew);
    if (isnew) {
      int slot = m + __popc(nm & lt);
      if (slot < kBigV) {
        float x, y, z, ev;
        vertex3<float>(big_plane(A, (int)a), big_plane(A, (int)b), H, x, y, z, ev);
        if (!(ev <= kRefineRel * (fabsf(x) + fabsf(y) + fabsf(z)))) {
          refine_vertex(A.pid[a], A.pid[b], hpid, c.me, c.lo, c.hi, sites, x, y, z, ev);
          ct.refv++;
        }
        A.nvp[slot] = make_float4(x, y, z, ev);
        A.nvt[slot] = btri(a, b, (uint32_t)h);
      }
    }
    m += __popc(nm);
  }
  if (counters) ct.newv += m;
  if (c.nv - k + m > kBigV) return CLIP_OVERFLOW;
  __syncwarp();
  // keep the inside vertices (in-place compaction), then append the new ones
  int kept = 0;
  for (int base = 0; base < c.nv; base += 32) {
    int i = base + (int)lane;
    bool keep = false;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    uint64_t T = 0;
    if (i < c.nv) {
      T = A.vt[i];
      keep = (T & kBigOut) == 0;
      if (keep) v = A.vp[i];
    }
    uint32_t km = __ballot_sync(FULL, keep);
    int dst = kept + __popc(km & lt);
    __syncwarp();
    if (keep) {
      A.vp[dst] = v;
      A.vt[dst] = T;
    }
    kept += __popc(km);
    __syncwarp();
  }
  for (int t = (int)lane; t < m; t += 32) {
    A.vp[kept + t] = A.nvp[t];
    A.vt[kept + t] = A.nvt[t];
  }
  c.nv = kept + m;
  __syncwarp();
  return CLIP_DONE;
}

// ---------------------------------------------------------------- queue
__device__ inline bool big_push(BigCell& c, const BigArena& A, float lb, int ref, int occ) {
  if (c.qn >= kBigQ) return false;
  if (lane_id() == 0) {
    A.qlb[c.qn] = lb;
    A.qref[c.qn] = ref;
    A.qocc[c.qn] = occ | (c.seq << 8);
  }
  c.qn++;
  c.seq++;
  __syncwarp();
  return true;
}

// Pop the best entry still valid under the current bounds; entries that
// fail the re-test are dropped, the popped slot takes the last entry
// (App. A.5).
__device__ inline bool big_pop(BigCell& c, const BigArena& A, int cull_mode, int traversal, int& ref) {
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
      lb = A.qlb[i];
      rf = A.qref[i];
      oc = A.qocc[i];
      float R = A.rtab[oc & 63];
      ok = cull_mode == 2 || !(lb > R * (1.0f + kCullPad));
      key = traversal == 0 ? f2o(lb - R) : (0xfffffffeu - (uint32_t)(oc >> 8));
    }
    uint32_t km = __ballot_sync(FULL, ok);
    int dst = live + __popc(km & lt);
    __syncwarp();
    if (ok) {
      A.qlb[dst] = lb;
      A.qref[dst] = rf;
      A.qocc[dst] = oc;
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
  if (mn == 0xffffffffu || live == 0) return false;
  int idx = (int)__reduce_min_sync(FULL, bestk == mn ? (uint32_t)besti : 0x7fffffffu);
  ref = A.qref[idx];
  __syncwarp();
  if (lane == 0) {
    int last = c.qn - 1;
    A.qlb[idx] = A.qlb[last];
    A.qref[idx] = A.qref[last];
    A.qocc[idx] = A.qocc[last];
  }
  c.qn--;
  __syncwarp();
  return true;
}

// Fill the pair hash with every vertex's three directed pairs -> vertex.
__device__ inline uint32_t big_hash_vertices(const BigCell& c, const BigArena& A) {
  uint32_t hs = hash_size(3 * c.nv);
  hash_clear(A, hs);
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    uint64_t T = A.vt[i];
#pragma unroll
    for (int r = 0; r < 3; r++) hash_insert(A, bpair(T, r), i, hs - 1);
  }
  __syncwarp();
  return hs - 1;
}

}  // namespace vd
