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
//
// Cells of large-weight sites reach thousands of vertices while almost all
// of their candidates (>99% on log-normal weights) cut nothing; each such
// candidate would otherwise test every vertex. The vertex array is therefore
// covered by chunk boxes (32 consecutive vertices each, with their largest
// error bound), rebuilt after every clip, and the read-only first pass tests
// a chunk's vertices only when the plane reaches the chunk's box. To keep
// the chunks compact, the vertex array of a large polytope is re-sorted after
// clips by the cube-map cell of its direction from the polytope's box centre
// (6 faces x 8 x 8 cells, Morton order within a face), so a chunk is a small
// patch of the surface and a plane that passes close to the polytope reaches
// the boxes of only a few patches.
//
// Vertex slots are not compacted after a clip: the new vertices of a clip
// take the slots of the vertices it removed (which lie where the new ones
// appear), extra ones come from a stack of free slots or the end of the
// array, and unused slots become dead (NaN position, which every sign test
// reads as inside and every box ignores). A clip therefore reads and writes
// only the chunks its plane reaches and refreshes only their boxes. The
// array is re-sorted, dropping dead slots, once the vertices placed outside
// their neighbours' chunks since the last sort pass 1/16 of the polytope.
#pragma once

#include "vd_clip.cuh"

namespace vd {

constexpr int kBigV = 16384;   // vertices per cell
constexpr int kBigP = 8192;    // planes per cell
constexpr int kBigQ = 8192;    // queue entries
constexpr int kBigH = 65536;   // pair-hash slots (power of two)
constexpr int kBigC = kBigV / 32;  // chunk boxes
constexpr int kBigGc = (kBigP * 85) / 100;
constexpr uint64_t kTriMask = 0x0000ffffffffffffull;
constexpr uint64_t kBigDead = kTriMask;  // triplet of a dead slot
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
  int4* q;  // best-first queue: 32-ary min-heap of (key, lb, ref, occ)
  uint32_t* hkey;
  int* hval;
  float* acc;
  float* rtab;  // [64] cell radius per occupied-octant mask
  float4* cb;   // [2 kBigC] chunk q: cb[2q] = (lo, max error), cb[2q+1] = (hi, 0)
  int* fs;      // [kBigV] free-slot stack
  int* os;      // [kBigV] slots of the vertices a clip removes
  // shared memory of the warp
  float4* hs;      // [32] staged candidate planes (n, b)
  float* hse;      // [32] their error bounds
  int* hid;        // [32] their sites
  float* hord;     // [32] their clip order key (plane offset)
  uint32_t* hist;  // [kDirBins] direction-bin counts / cursors
  uint32_t* cdirty;  // [kBigC / 32] chunks whose box is stale
  struct HelpBoard* hb;  // the block's helping board (forward large-cell kernel only)
  int* err;              // device error word
  int* stall;            // test hook (see help_drain), or nullptr
};

constexpr int kDirBins = 6 * 64;
// Polytopes of more vertices than this are kept in direction-bin order.
constexpr int kSortMin = 128;

// Shared memory per warp of the large-cell kernels.
constexpr size_t kBigSmemPerWarp = 32 * 16 + 3 * 32 * 4 + kDirBins * 4 + kBigC / 8;

__host__ __device__ inline size_t big_arena_bytes() {
  size_t b = 64 * 4;
  b += (size_t)kBigP * (16 + 4 + 4 + 4);
  b += (size_t)kBigV * (16 + 8 + 8 + 16 + 8);
  b += (size_t)kBigQ * 16;
  b += (size_t)kBigH * 8;
  b += (size_t)kBigP * 10 * 4;
  b += 64 * 4 + (size_t)kBigC * 32;
  b += (size_t)kBigV * 8;
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
  A.q = (int4*)p;
  p += (size_t)kBigQ * 16;
  A.hkey = (uint32_t*)p;
  p += (size_t)kBigH * 4;
  A.hval = (int*)p;
  p += (size_t)kBigH * 4;
  A.acc = (float*)p;
  p += (size_t)kBigP * 10 * 4;
  A.rtab = (float*)p;
  p += 64 * 4;
  A.cb = (float4*)p;
  p += (size_t)kBigC * 32;
  A.fs = (int*)p;
  p += (size_t)kBigV * 4;
  A.os = (int*)p;
  extern __shared__ __align__(16) char big_smem[];
  char* w = big_smem + (size_t)(threadIdx.x >> 5) * kBigSmemPerWarp;
  A.hs = (float4*)w;
  A.hse = (float*)(w + 32 * 16);
  A.hid = (int*)(w + 32 * 16 + 32 * 4);
  A.hord = (float*)(w + 32 * 16 + 2 * 32 * 4);
  A.hist = (uint32_t*)(w + 32 * 16 + 3 * 32 * 4);
  A.cdirty = (uint32_t*)(w + 32 * 16 + 3 * 32 * 4 + kDirBins * 4);
  A.hb = nullptr;
  A.err = nullptr;
  A.stall = nullptr;
  return A;
}

// Large-cell tape record (the forward's polytope of a cell that left the
// register path, so that the adjoint restores it instead of re-clipping):
// int4 (nv, npl, 0, 0), nv float4 vertices, nv uint64 plane triplets, npl
// plane ids; 16-byte aligned. The site's regular tape header then reads
// (-2, npl, low and high 32 bits of the record's byte offset).
constexpr long long kBigTapePerSite = 128;  // pool bytes reserved per site
__host__ __device__ inline long long big_tape_bytes(int nv, int npl) {
  return (16 + 24LL * nv + 4LL * npl + 15) & ~15LL;
}

struct BigCell {
  float4 me;
  float lo[3], hi[3];
  float alo[3], ahi[3];
  float sc[3], srad;
  float em;      // largest vertex error bound
  int nv;        // vertex slots in use (live and dead)
  int nlive;     // live vertices
  int nfree;     // dead slots on the free-slot stack
  int unsorted;  // vertices placed away from their clip's chunks since the last sort
  int npl, qn, seq;
  int nst;  // candidate planes staged in A.hs for the next filter
  bool dirty;
  bool fp64;  // FP64 re-evaluation of ambiguous predicates, vertices and volumes
};

__device__ __forceinline__ bool bdead(uint64_t T) { return (T & kTriMask) == kTriMask; }

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

// Cube-map cell of direction (dx, dy, dz): face * 64 + Morton(iu, iv) on an
// 8 x 8 grid of the face.
__device__ __forceinline__ uint32_t dir_bin(float dx, float dy, float dz) {
  const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
  uint32_t f;
  float m, a, b;
  if (ax >= ay && ax >= az) {
    f = dx >= 0.0f ? 0u : 1u;
    m = ax;
    a = dy;
    b = dz;
  } else if (ay >= az) {
    f = dy >= 0.0f ? 2u : 3u;
    m = ay;
    a = dz;
    b = dx;
  } else {
    f = dz >= 0.0f ? 4u : 5u;
    m = az;
    a = dx;
    b = dy;
  }
  const float inv = m > 0.0f ? 4.0f / m : 0.0f;
  const uint32_t iu = (uint32_t)min(7, max(0, (int)fmaf(a, inv, 4.0f)));
  const uint32_t iv = (uint32_t)min(7, max(0, (int)fmaf(b, inv, 4.0f)));
  uint32_t mo = 0;
#pragma unroll
  for (int k = 0; k < 3; k++) mo |= (((iu >> k) & 1u) << (2 * k)) | (((iv >> k) & 1u) << (2 * k + 1));
  return f * 64u + mo;
}

// Stable counting sort of the live vertices by direction bin about the box
// centre (c.sc), through the staging arrays nvp / nvt; dead slots are
// dropped (bins == 1: compaction only, order kept).
__device__ inline void big_sort_vertices(BigCell& c, const BigArena& A, bool bins = true) {
  const unsigned lane = lane_id(), lt = lanemask_lt();
  for (int b = (int)lane; b < kDirBins; b += 32) A.hist[b] = 0;
  __syncwarp();
  for (int i = (int)lane; i < c.nv; i += 32) {
    const float4 v = A.vp[i];
    if (!bdead(A.vt[i])) atomicAdd(&A.hist[bins ? dir_bin(v.x - c.sc[0], v.y - c.sc[1], v.z - c.sc[2]) : 0u], 1u);
  }
  __syncwarp();
  // exclusive scan: lane l owns bins [12 l, 12 l + 12)
  {
    constexpr int per = kDirBins / 32;
    uint32_t loc[per], sum = 0;
#pragma unroll
    for (int k = 0; k < per; k++) {
      loc[k] = A.hist[per * lane + k];
      sum += loc[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, incl, o);
      if ((int)lane >= o) incl += t;
    }
    uint32_t run = incl - sum;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < per; k++) {
      A.hist[per * lane + k] = run;
      run += loc[k];
    }
  }
  __syncwarp();
  for (int base = 0; base < c.nv; base += 32) {
    const int i = base + (int)lane;
    const bool in = i < c.nv;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    uint64_t T = 0;
    uint32_t b = 0xffffffffu;
    if (in) {
      v = A.vp[i];
      T = A.vt[i];
      if (!bdead(T)) b = bins ? dir_bin(v.x - c.sc[0], v.y - c.sc[1], v.z - c.sc[2]) : 0u;
    }
    const uint32_t peers = __match_any_sync(FULL, b);
    const int pos = b != 0xffffffffu ? (int)A.hist[b] + __popc(peers & lt) : 0;
    __syncwarp();
    if (b != 0xffffffffu) {
      A.nvp[pos] = v;
      A.nvt[pos] = T;
      if ((peers & lt) == 0) A.hist[b] += __popc(peers);
    }
    __syncwarp();
  }
  c.nv = c.nlive;
  c.nfree = 0;
  c.unsorted = 0;
  for (int i = (int)lane; i < c.nv; i += 32) {
    A.vp[i] = A.nvp[i];
    A.vt[i] = A.nvt[i];
  }
  __syncwarp();
}

// Drop dead slots (order kept): the array is dense afterwards, as the
// volume and gradient passes expect.
__device__ inline void big_compact(BigCell& c, const BigArena& A) {
  if (c.nlive != c.nv) big_sort_vertices(c, A, false);
}

// Chunk boxes of the current vertex array (exact min / max of the stored
// FP32 positions).
__device__ inline void big_chunk_box(const BigCell& c, const BigArena& A, int q) {
  {
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY, em = 0.0f;
    const int i1 = min(c.nv, 32 * q + 32);
#pragma unroll 8
    for (int i = 32 * q; i < i1; i++) {
      const float4 v = A.vp[i];
      lx = fminf(lx, v.x);
      ly = fminf(ly, v.y);
      lz = fminf(lz, v.z);
      hx = fmaxf(hx, v.x);
      hy = fmaxf(hy, v.y);
      hz = fmaxf(hz, v.z);
      em = fmaxf(em, v.w);
    }
    A.cb[2 * q] = make_float4(lx, ly, lz, em);
    A.cb[2 * q + 1] = make_float4(hx, hy, hz, 0.0f);
  }
}

__device__ inline void big_chunk_boxes(const BigCell& c, const BigArena& A) {
  const int nch = (c.nv + 31) >> 5;
  for (int q = (int)lane_id(); q < nch; q += 32) big_chunk_box(c, A, q);
  for (int w = (int)lane_id(); w < kBigC / 32; w += 32) A.cdirty[w] = 0;
  __syncwarp();
}

// Refresh the boxes of the chunks marked in A.cdirty.
__device__ inline void big_dirty_boxes(const BigCell& c, const BigArena& A) {
  const int nch = (c.nv + 31) >> 5;
  for (int w = 0; w < (nch + 31) >> 5; w++) {
    const uint32_t bits = A.cdirty[w];
    if (bits == 0) continue;
    const int q = 32 * w + (int)lane_id();
    if ((bits >> lane_id()) & 1u) big_chunk_box(c, A, q);
    __syncwarp();
    if (lane_id() == 0) A.cdirty[w] = 0;
  }
  __syncwarp();
}

// May plane H leave a vertex of the chunk with box (lo, hi) outside or
// ambiguous? S = max over the box of n.x - b bounds n.v - b for every
// vertex v in it; the FP32 evaluations of S and of a vertex's sign test
// each round by at most 4u (|n|.max|x| + |b|), so a chunk whose S stays
// below -(2 (emax + e_H) + 8u (...)) holds only vertices the sign test
// classifies as certainly inside.
__device__ __forceinline__ bool chunk_may_cut(const PlaneT<float>& H, float4 lo, float4 hi) {
  const float u = Num<float>::u;
  const float sx = H.nx >= 0.0f ? hi.x : lo.x, sy = H.ny >= 0.0f ? hi.y : lo.y, sz = H.nz >= 0.0f ? hi.z : lo.z;
  const float S = fmaf(H.nx, sx, fmaf(H.ny, sy, fmaf(H.nz, sz, -H.b)));
  const float m1 = fabsf(H.nx) * fmaxf(fabsf(lo.x), fabsf(hi.x)) + fabsf(H.ny) * fmaxf(fabsf(lo.y), fabsf(hi.y)) +
                   fabsf(H.nz) * fmaxf(fabsf(lo.z), fabsf(hi.z)) + fabsf(H.b);
  return !(S < -(2.0f * (lo.w + H.e) + 8.0f * u * m1));
}

// Polytopes of at most this many chunks are scanned without the box stage.
constexpr int kBoxStage = 2;
// Chunk ranges of at most this many chunks test their boxes one lane per plane.
constexpr int kByPlaneChunks = 12;

// Batch filter: which of the k <= 32 planes staged in A.hs / A.hse may
// cut the polytope (some vertex outside or ambiguous)? Bit t of the result
// stands for plane t. Each vertex chunk is loaded once for all planes whose
// test reaches its box. A plane that leaves every vertex certainly inside
// also leaves every later (clipped, smaller) polytope of the cell inside, so
// the caller drops it for good.
// The staged planes (hs, hse) of mask m, four per step so that their
// shared-memory loads and tests overlap; f(t, H) is called for each.
template <typename F>
__device__ __forceinline__ void for_staged_planes(const float4* hs, const float* hse, uint32_t m, F f) {
  while (m) {
    int t[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      t[u] = m ? __ffs(m) - 1 : -1;
      m &= m ? m - 1 : 0u;
    }
    PlaneT<float> H[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int tt = t[u] < 0 ? t[0] : t[u];
      const float4 h = hs[tt];
      H[u].nx = h.x;
      H[u].ny = h.y;
      H[u].nz = h.z;
      H[u].b = h.w;
      H[u].e = hse[tt];
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (t[u] >= 0) f(t[u], H[u]);
  }
}

// Which of the planes in `open` (staged at hs / hse) leave a vertex of the
// chunks [q0, q1) outside or ambiguous? Chunk boxes are tested first when
// `boxes`; each flagged chunk's vertices are loaded once for all the planes
// whose test reaches its box.
__device__ inline uint32_t filter_chunks(const float4* vp, const float4* cb, int nv, int q0, int q1,
                                         const float4* hs, const float* hse, uint32_t open, bool boxes,
                                         long long& tested, bool group = false) {
  const unsigned lane = lane_id();
  uint32_t cuts = 0;
  // a helping group (a few chunks of another warp's polytope) tests its
  // boxes with one lane per staged plane, so that all lanes work; a warp's
  // own filter takes one lane per chunk and loops over the open planes
  const bool by_plane = group && boxes && q1 - q0 <= kByPlaneChunks;
  PlaneT<float> Hl;
  Hl.nx = Hl.ny = Hl.nz = Hl.b = Hl.e = 0.0f;
  if (by_plane && ((open >> lane) & 1u)) {
    const float4 h = hs[lane];
    Hl.nx = h.x;
    Hl.ny = h.y;
    Hl.nz = h.z;
    Hl.b = h.w;
    Hl.e = hse[lane];
  }
  for (int cbase = q0; cbase < q1 && open; cbase += 32) {
    const int q = cbase + (int)lane;
    uint32_t fl = 0;
    if (by_plane) {
      const int m = min(32, q1 - cbase);
      for (int r = 0; r < m; r++) {
        const float4 lo = cb[2 * (cbase + r)], hi = cb[2 * (cbase + r) + 1];
        const uint32_t b = __ballot_sync(FULL, ((open >> lane) & 1u) && chunk_may_cut(Hl, lo, hi));
        if ((int)lane == r) fl = b;
      }
    } else if (q < q1) {
      if (!boxes) {
        fl = open;
      } else {
        const float4 lo = cb[2 * q], hi = cb[2 * q + 1];
        for_staged_planes(hs, hse, open, [&](int t, const PlaneT<float>& H) {
          if (chunk_may_cut(H, lo, hi)) fl |= 1u << t;
        });
      }
    }
    uint32_t U = __ballot_sync(FULL, fl != 0);
    while (U && open) {
      // up to four flagged chunks per step, their vertex loads in flight together
      int qs[4];
      uint32_t pms[4];
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        qs[u] = U ? __ffs(U) - 1 : -1;
        U &= U ? U - 1 : 0u;
        pms[u] = __shfl_sync(FULL, fl, qs[u] < 0 ? 0 : qs[u]) & open;
        if (qs[u] < 0) pms[u] = 0;
        const int i = 32 * (cbase + (qs[u] < 0 ? 0 : qs[u])) + (int)lane;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pms[u] && i < nv) v[u] = vp[i];
      }
      uint32_t outm = 0;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int i = 32 * (cbase + (qs[u] < 0 ? 0 : qs[u])) + (int)lane;
        if (i < nv) {
          const float4 w = v[u];
          for_staged_planes(hs, hse, pms[u], [&](int t, const PlaneT<float>& H) {
            const float s = side<float>(H, w.x, w.y, w.z);
            if (s > 0.0f || ambiguous<float>(s, w.w, H.e)) outm |= 1u << t;
          });
        }
        tested += 32 * __popc(pms[u]);
      }
      outm = __reduce_or_sync(FULL, outm);
      cuts |= outm;
      open &= ~outm;
    }
  }
  return cuts;
}

// ---------------------------------------------------------------- helping
//
// Warps of a large-cell block that have run out of cells help the others'
// batch filters (the dominant step of cells with thousands of vertices).
// The owner posts a request (its planes stay in its shared memory, its
// vertex and chunk arrays in its arena); every warp of the block, the owner
// included, claims groups of kHelpGroup chunks by compare-and-swap on a
// counter tagged with the request's generation, ORs the planes it finds
// cutting into the request and then counts the chunks done; the owner
// closes the request once every chunk is done. A claim succeeds only while
// its generation is open and chunks remain, and the owner cannot close
// before every claimed group is counted, so a helper never works on a
// request that was closed or re-opened under it. Waits are bounded: a wait
// that runs out sets VD_ERR_TIMEOUT and returns.
struct HelpReq {
  int seq;        // odd while open
  int next;       // generation << 20 | next unclaimed chunk
  int done;       // chunks finished
  unsigned cuts;  // planes found cutting
  int nch, k, nv, pad;
  const float4* vp;
  const float4* cb;
  const float4* hs;
  const float* hse;
};
struct HelpBoard {
  HelpReq req[kBigWarpsPerBlock];
  int live;  // warps of the block still building their own cells
};
constexpr int kHelpMinChunks = 32;  // filters over fewer chunks run alone
constexpr int kHelpGroup = 8;       // chunks per claim
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ int vload(const int* p) { return *(const volatile int*)p; }

__device__ inline void set_error_timeout(const BigArena& A) {
  if (A.err) atomicCAS(A.err, 0, VD_ERR_TIMEOUT);
}

// Lane 0: claim the next group of request r (generation gen); -1 if none.
__device__ inline int help_claim(HelpReq& r, int gen, int nch) {
  int old = vload(&r.next);
  while (true) {
    if ((old >> 20) != gen) return -1;
    const int idx = old & 0xfffff;
    if (idx >= nch) return -1;
    const int prev = atomicCAS(&r.next, old, old + kHelpGroup);
    if (prev == old) return idx;
    old = prev;
  }
}

// Work on request r through its groups; returns the number of groups done
// once none is left to claim. Test hook: while the token `stall` is armed,
// the first group claimed is never counted, so its owner's bounded wait runs
// out and reports VD_ERR_TIMEOUT (nothing else waits on that count).
__device__ inline int help_drain(HelpReq& r, int gen, long long& tested, int* stall) {
  const unsigned lane = lane_id();
  int groups = 0;
  while (true) {
    int q0 = -1;
    if (lane == 0) q0 = help_claim(r, gen, vload(&r.nch));
    q0 = __shfl_sync(FULL, q0, 0);
    if (q0 < 0) return groups;
    groups++;
    // the request is open and unchanged while a claimed group is uncounted
    const int nch = vload(&r.nch), k = vload(&r.k), nv = vload(&r.nv);
    const float4* vp = r.vp;
    const float4* cb = r.cb;
    const float4* hs = r.hs;
    const float* hse = r.hse;
    const uint32_t open = (k >= 32 ? FULL : ((1u << k) - 1u)) & ~(uint32_t)vload((const int*)&r.cuts);
    const int q1 = min(nch, q0 + kHelpGroup);
    const uint32_t cm = filter_chunks(vp, cb, nv, q0, q1, hs, hse, open, true, tested, true);
    if (lane == 0) {
      if (cm) atomicOr(&r.cuts, cm);
      __threadfence_block();
      const bool skip = stall != nullptr && atomicExch(stall, 0) != 0;
      if (!skip) atomicAdd(&r.done, q1 - q0);
    }
    __syncwarp();
  }
}

// Batch filter: which of the k <= 32 planes staged in A.hs / A.hse may
// cut the polytope (some vertex outside or ambiguous)? Bit t of the result
// stands for plane t. A plane that leaves every vertex certainly inside
// also leaves every later (clipped, smaller) polytope of the cell inside, so
// the caller drops it for good.
__device__ inline uint32_t big_filter(const BigCell& c, const BigArena& A, int k, Counters& ct, bool counters) {
  const unsigned lane = lane_id();
  const uint32_t open = k >= 32 ? FULL : ((1u << k) - 1u);
  long long tested = 0;
  const int nch = (c.nv + 31) >> 5;
  uint32_t cuts;
  // post a request only when some warp of the block has no cell of its own
  bool share = A.hb != nullptr && nch >= kHelpMinChunks;
  if (share) share = __shfl_sync(FULL, vload(&A.hb->live), 0) < (int)(blockDim.x >> 5);
  if (!share) {
    cuts = filter_chunks(A.vp, A.cb, c.nv, 0, nch, A.hs, A.hse, open, nch > kBoxStage, tested);
  } else {
    HelpReq& r = A.hb->req[threadIdx.x >> 5];
    int gen = 0;
    if (lane == 0) {
      gen = ((vload(&r.seq) >> 1) + 1) & 0x7ff;
      r.nch = nch;
      r.k = k;
      r.nv = c.nv;
      r.vp = A.vp;
      r.cb = A.cb;
      r.hs = A.hs;
      r.hse = A.hse;
      r.done = 0;
      r.cuts = 0;
      r.next = gen << 20;
      __threadfence_block();  // the arena's vertices and boxes and the request fields before the opening
      atomicAdd(&r.seq, 1);
    }
    gen = __shfl_sync(FULL, gen, 0);
    help_drain(r, gen, tested, A.stall);
    if (lane == 0) {
      long long it = 0;
      while (vload(&r.done) < nch) {
        __nanosleep(32);
        if (++it > kWaitLimit) {
          set_error_timeout(A);
          break;
        }
      }
      __threadfence_block();
    }
    __syncwarp();
    cuts = (uint32_t)vload((const int*)&r.cuts);
    cuts = __shfl_sync(FULL, cuts, 0);
    if (lane == 0) atomicAdd(&r.seq, 1);
    __syncwarp();
  }
  if (counters) ct.vtests += tested;
  return cuts;
}

// A warp that has no cell left helps the block's open requests until every
// warp of the block has finished its own cells (bounded wait).
__device__ inline void big_help(const BigArena& A, long long& tested) {
  const unsigned lane = lane_id();
  const int me = (int)(threadIdx.x >> 5);
  if (lane == 0) atomicSub(&A.hb->live, 1);
  long long it = 0;
  while (true) {
    bool worked = false;
    for (int w = 0; w < kBigWarpsPerBlock; w++) {
      if (w == me) continue;
      HelpReq& r = A.hb->req[w];
      int s = vload(&r.seq);
      s = __shfl_sync(FULL, s, 0);
      if (!(s & 1)) continue;
      if (help_drain(r, ((s >> 1) + 1) & 0x7ff, tested, A.stall) > 0) worked = true;
    }
    if (worked) continue;
    int live = vload(&A.hb->live);
    live = __shfl_sync(FULL, live, 0);
    if (live <= 0) break;
    __nanosleep(256);
    if (++it > kWaitLimit) break;
  }
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
  c.em = em;
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
  c.nlive = 8;
  c.nfree = 0;
  c.unsorted = 0;
  c.nst = 0;
  c.npl = 6;
  c.qn = 0;
  c.seq = 0;
  c.dirty = false;
  __syncwarp();
  big_chunk_boxes(c, A);
  big_aabb(c, A, cull_mode);
}

// Mark the planes referenced by the vertices in A.flag (1 / 0).
__device__ inline void big_mark_planes(const BigCell& c, const BigArena& A) {
  for (int p = (int)lane_id(); p < c.npl; p += 32) A.flag[p] = 0;
  __syncwarp();
  for (int i = (int)lane_id(); i < c.nv; i += 32) {
    uint64_t T = A.vt[i];
    if (bdead(T)) continue;
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
    if (!bdead(T)) A.vt[i] = btri(A.flag[bfield(T, 0)], A.flag[bfield(T, 1)], A.flag[bfield(T, 2)]);
  }
  c.npl = alive;
  __syncwarp();
}

static __device__ __noinline__ bool big_resolve64(const BigArena& A, uint64_t tri, int hpid, float4 me, const float* lo,
                                           const float* hi, const float4* __restrict__ sites, long long& amb) {
  const Plane64u P0 = plane64u(A.pid[bfield(tri, 0)], me, lo, hi, sites);
  const Plane64u P1 = plane64u(A.pid[bfield(tri, 1)], me, lo, hi, sites);
  const Plane64u P2 = plane64u(A.pid[bfield(tri, 2)], me, lo, hi, sites);
  const Plane64u H = plane64u(hpid, me, lo, hi, sites);
  bool a = false;
  const bool out = side64u(P0, P1, P2, H, a);
  if (a) amb++;
  return out;
}

// Clip by plane H of site hpid (App. B), memory-resident form. `filtered`:
// the batch filter found that the plane may cut this cell (a vertex outside
// or ambiguous), so the read-only pass that screens candidates which cut
// nothing is skipped; the classifying pass alone still returns CLIP_NONE
// when earlier clips left nothing outside.
static __device__ int big_clip(BigCell& c, const BigArena& A, const PlaneT<float>& H, int hpid,
                        const float4* __restrict__ sites, Counters& ct, bool counters, bool filtered = false) {
  const unsigned lane = lane_id(), lt = lanemask_lt();
  if (c.npl >= kBigGc) big_gc(c, A);
  if (c.npl >= kBigP) return CLIP_OVERFLOW;
  // read-only first pass over the chunks whose box the plane reaches; most
  // candidates cut nothing and end here without writes
  if (!filtered) {
    bool any = false;
    const int nch = (c.nv + 31) >> 5;
    long long tested = 0;
    for (int cbase = 0; cbase < nch && !any; cbase += 32) {
      const int q = cbase + (int)lane;
      bool f = q < nch;
      if (f && nch > kBoxStage) f = chunk_may_cut(H, A.cb[2 * q], A.cb[2 * q + 1]);
      uint32_t fm = __ballot_sync(FULL, f);
      while (fm && !any) {
        // up to four flagged chunks per step, their loads in flight together
        int qs[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          qs[u] = fm ? cbase + __ffs(fm) - 1 : -1;
          fm &= fm - 1;
        }
        bool o = false;
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int i = 32 * qs[u] + (int)lane;
          if (qs[u] >= 0 && i < c.nv) {
            float4 v = A.vp[i];
            float s = side<float>(H, v.x, v.y, v.z);
            bool out = s > 0.0f;
            if (ambiguous<float>(s, v.w, H.e)) out = true;  // settled in FP64 by the marking pass
            o = o || out;
          }
          tested += qs[u] >= 0 ? 32 : 0;
        }
        any = __any_sync(FULL, o);
      }
    }
    if (counters) ct.vtests += tested;
    if (!any) return CLIP_NONE;
  }
  // classify the vertices of the chunks the plane reaches; list the outside
  // ones' triplets (otri) and slots (os)
  int k = 0;
  {
    const int nch = (c.nv + 31) >> 5;
    for (int cbase = 0; cbase < nch; cbase += 32) {
      const int q = cbase + (int)lane;
      bool f = q < nch;
      if (f && nch > kBoxStage) f = chunk_may_cut(H, A.cb[2 * q], A.cb[2 * q + 1]);
      uint32_t fm = __ballot_sync(FULL, f);
      while (fm) {
        int qs[4];
        float4 v[4];
        uint64_t T[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          qs[u] = fm ? cbase + __ffs(fm) - 1 : -1;
          fm &= fm ? fm - 1 : 0u;
          const int i = 32 * qs[u] + (int)lane;
          v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          T[u] = kBigDead;
          if (qs[u] >= 0 && i < c.nv) {
            v[u] = A.vp[i];
            T[u] = A.vt[i];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int i = 32 * qs[u] + (int)lane;
          bool out = false;
          if (!bdead(T[u])) {
            float s = side<float>(H, v[u].x, v[u].y, v[u].z);
            out = s > 0.0f;
            if (c.fp64 && ambiguous<float>(s, v[u].w, H.e)) {
              ct.fp64++;
              out = big_resolve64(A, T[u], hpid, c.me, c.lo, c.hi, sites, ct.fp64amb);
            }
          }
          uint32_t m = __ballot_sync(FULL, out);
          if (out) {
            A.otri[k + __popc(m & lt)] = T[u];
            A.os[k + __popc(m & lt)] = i;
          }
          k += __popc(m);
        }
      }
    }
  }
  __syncwarp();
  if (k == 0) return CLIP_NONE;
  if (k == c.nlive) return CLIP_EMPTY;
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
        if (c.fp64 && !(ev <= kRefineRel * (fabsf(x) + fabsf(y) + fabsf(z)))) {
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
  if (m > k + c.nfree + (kBigV - c.nv)) return CLIP_OVERFLOW;
  __syncwarp();
  // new vertex t takes the slot of removed vertex t, then free slots, then
  // slots at the end; removed slots left over become dead and free
  const int from_free = min(max(m - k, 0), c.nfree);
  for (int t = (int)lane; t < max(m, k); t += 32) {
    int slot;
    if (t < k)
      slot = A.os[t];
    else if (t - k < from_free)
      slot = A.fs[c.nfree - 1 - (t - k)];
    else
      slot = c.nv + (t - k - from_free);
    if (t < m) {
      A.vp[slot] = A.nvp[t];
      A.vt[slot] = A.nvt[t];
    } else {
      A.vp[slot] = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000), 0.0f);
      A.vt[slot] = kBigDead;
    }
    atomicOr(&A.cdirty[slot >> 10], 1u << ((slot >> 5) & 31));
  }
  __syncwarp();
  if (m < k) {
    for (int t = m + (int)lane; t < k; t += 32) A.fs[c.nfree + (t - m)] = A.os[t];
    c.nfree += k - m;
  } else {
    c.nfree -= from_free;
    c.nv += m - k - from_free;
    c.unsorted += m - k;
  }
  c.nlive += m - k;
  __syncwarp();
  if (c.nlive > kSortMin && c.unsorted > max(64, c.nlive >> 4)) {
    big_sort_vertices(c, A);
    big_chunk_boxes(c, A);
  } else {
    big_dirty_boxes(c, A);
  }
  return CLIP_DONE;
}

// ---------------------------------------------------------------- queue
__device__ inline bool big_push(BigCell& c, const BigArena& A, float lb, float key, int traversal, int ref, int occ) {
  if (c.qn >= kBigQ) return false;
  if (lane_id() == 0) {
    // sift up from the new leaf
    const uint32_t k = traversal == 0 ? f2o(key) : 0xfffffffeu - (uint32_t)c.seq;
    const int4 e = make_int4((int)k, __float_as_int(lb), ref, occ | (c.seq << 8));
    int i = c.qn;
    while (i > 0) {
      const int p = (i - 1) >> 5;
      const int4 pe = A.q[p];
      if ((uint32_t)pe.x <= k) break;
      A.q[i] = pe;
      i = p;
    }
    A.q[i] = e;
  }
  c.qn++;
  c.seq++;
  __syncwarp();
  return true;
}

// Pop the entry of least key (the key is fixed when the entry is pushed);
// an entry that fails the re-test under the current bounds is dropped and
// the next one taken. The heap is 32-ary, so each level of the sift-down is
// one coalesced load of the 32 children and a warp minimum.
__device__ inline bool big_pop(BigCell& c, const BigArena& A, int cull_mode, int& ref) {
  const unsigned lane = lane_id();
  while (c.qn > 0) {
    const int4 top = A.q[0];
    c.qn--;
    const int4 last = A.q[c.qn];
    int i = 0;
    while (true) {
      const int c0 = 32 * i + 1;
      if (c0 >= c.qn) break;
      const int j = c0 + (int)lane;
      int4 ch = make_int4(-1, 0, 0, 0);
      if (j < c.qn) ch = A.q[j];
      const uint32_t mn = __reduce_min_sync(FULL, (uint32_t)ch.x);
      if (mn >= (uint32_t)last.x) break;
      const int src = __ffs(__ballot_sync(FULL, j < c.qn && (uint32_t)ch.x == mn)) - 1;
      __syncwarp();
      if ((int)lane == src) A.q[i] = ch;
      i = c0 + src;
    }
    __syncwarp();
    if (lane == 0 && c.qn > 0) A.q[i] = last;
    __syncwarp();
    const float lb = __int_as_float(top.y);
    const float R = A.rtab[top.w & 63];
    if (cull_mode == 2 || !(lb > R * (1.0f + kCullPad))) {
      ref = top.z;
      return true;
    }
  }
  return false;
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
