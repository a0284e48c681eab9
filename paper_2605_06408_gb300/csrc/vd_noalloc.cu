// vd_noalloc.cu -- vd_cells_noalloc: cells of a small point set without any
// device allocation.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator hooks, real-time or safety-critical
// loops that forbid allocation after start-up, and callers that must not
// create a context workspace at all. For them this entry point keeps all of
// its scratch (the packed sites, a duplicate mask, a work counter and a
// status block) in one file-scope device array of fixed size, and writes
// only into the buffers the caller passes.
//
// It is a variant of the fused cell kernel: every other site is a candidate
// (no BVH, so no sort or tree buffers are needed), taken 32 at a time like a
// leaf and culled by the same AABB / sphere tests, then clipped with the same
// register-resident clipping. Cells that outgrow the register capacity, or
// have more than VD_NOALLOC_ROW neighbours, are reported in the status word
// instead of moving to the large-cell path (which needs an arena).
#include <cuda.h>  // CUcontext / CUresult types of the two driver calls looked up below

#include <mutex>

#include "vd_clip.cuh"

namespace vd {
namespace {

constexpr int kNaMaxSites = VD_NOALLOC_MAX_SITES;
constexpr int kNaRow = VD_NOALLOC_ROW;
constexpr int kNaVpl = 4;
constexpr int kNaPcap = 128;
constexpr int kNaWarps = 4;

struct NoAllocScratch {
  float4 sites[kNaMaxSites];         // packed (x, y, z, w), by site index
  float box[6];                      // lo[3], hi[3]
  unsigned char loser[kNaMaxSites];  // an exact duplicate site beats this one
  int work;                          // persistent-grid work counter
  int error;                         // first device-side error
};

// The scratch array itself. In host code `g_scratch` names a host-side
// stand-in, not device memory: the device address comes from
// cudaGetSymbolAddress (see scratch_on_device below).
static __device__ __align__(256) unsigned char g_scratch[sizeof(NoAllocScratch)];

using Smem = WarpSmem<kNaVpl, kNaPcap, 1>;
using CellT = Cell<kNaVpl, kNaPcap, 1>;

__global__ void na_pack_kernel(const float* __restrict__ xyz, const float* __restrict__ w, int n, vd_box box,
                               NoAllocScratch* S) {
  if (blockIdx.x == 0 && threadIdx.x < 6) S->box[threadIdx.x] = threadIdx.x < 3 ? box.lo[threadIdx.x] : box.hi[threadIdx.x - 3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    float wi = w ? w[i] : 0.0f;
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(wi))) atomicCAS(&S->error, 0, VD_ERR_INVALID_ARG);
    S->sites[i] = make_float4(x, y, z, wi);
    // duplicate rule: the larger weight, then the lower index, keeps the cell
    bool lose = false;
    for (int j = 0; j < n && !lose; j++) {
      if (j == i || xyz[3 * j] != x || xyz[3 * j + 1] != y || xyz[3 * j + 2] != z) continue;
      float wj = w ? w[j] : 0.0f;
      lose = wj > wi || (wj == wi && j < i);
    }
    S->loser[i] = lose ? 1 : 0;
  }
}

// A cell this entry point cannot hold (register capacity, or more than
// kNaRow neighbours): count -1, NaN volume and centroid, status word set.
__device__ inline void overflow_row(int i, int32_t* counts, float* vol, float* cen, NoAllocScratch* SC) {
  const float qnan = __int_as_float(0x7fc00000);
  counts[i] = -1;
  vol[i] = qnan;
  cen[3 * (size_t)i] = qnan;
  cen[3 * (size_t)i + 1] = qnan;
  cen[3 * (size_t)i + 2] = qnan;
  atomicCAS(&SC->error, 0, VD_ERR_CELL_OVERFLOW);
}

// One warp per cell, every other site a candidate.
__global__ void __launch_bounds__(32 * kNaWarps) na_cells_kernel(int n, int32_t* __restrict__ counts,
                                                                 int32_t* __restrict__ nbrs,
                                                                 float* __restrict__ vol, float* __restrict__ cen,
                                                                 NoAllocScratch* SC) {
  __shared__ Smem smem[kNaWarps];
  Smem& S = smem[threadIdx.x >> 5];
  const unsigned lane = lane_id(), lt = lanemask_lt();
  const float4* __restrict__ sites = SC->sites;
  if (lane == 0) S.ct = WarpCounters{};
  __syncwarp();
  while (true) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&SC->work, 1);
    i = __shfl_sync(FULL, i, 0);
    if (i >= n) break;
    CellT c;
    c.me = sites[i];
    c.box = SC->box;
    c.fp64 = true;
    bool empty = SC->loser[i] != 0, overflow = false;
    if (!empty) init_cell(c, S, 0);
    for (int base = 0; base < n && !empty && !overflow; base += 32) {
      const int j = base + (int)lane;
      bool keep = false;
      PlaneT<float> H;
      H.nx = H.ny = H.nz = H.b = H.e = 0.0f;
      float dkey = INFINITY;
      if (j < n && j != i && !SC->loser[j]) {
        float4 q = sites[j];
        float nx = q.x - c.me.x, ny = q.y - c.me.y, nz = q.z - c.me.z;
        float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
        if (nx == 0.0f && ny == 0.0f && nz == 0.0f) {
          // i is not a loser, so an exact duplicate j is one: implied plane
        } else {
          float beta = 0.5f * (nn + (c.me.w - q.w));
          keep = candidate_test(nx, ny, nz, nn, beta, c.me.w, q.w, c.alo, c.ahi, c.sc, c.srad, 0);
          if (keep) {
            H = site_plane<float>(c.me.x, c.me.y, c.me.z, c.me.w, q.x, q.y, q.z, q.w);
            dkey = H.b;
          }
        }
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
        if ((int)lane == src) keep = false;
        km &= ~(1u << src);
        int rc = clip_cell(c, S, Hb, base + src, sites, false);
        if (rc == CLIP_EMPTY) {
          empty = true;
          break;
        }
        if (rc == CLIP_OVERFLOW || rc == CLIP_OVF_PLANES) {
          overflow = true;
          break;
        }
        if (rc == CLIP_DONE) c.dirty = true;
      }
      if (c.dirty && !empty && !overflow) {
        recompute_aabb(c, S, 0);
        c.dirty = false;
      }
    }
    if (overflow) {
      if (lane == 0) overflow_row(i, counts, vol, cen, SC);
      continue;
    }
    if (empty) {
      if (lane == 0) {
        counts[i] = 0;
        vol[i] = 0.0f;
        cen[3 * (size_t)i] = c.me.x;
        cen[3 * (size_t)i + 1] = c.me.y;
        cen[3 * (size_t)i + 2] = c.me.z;
      }
      continue;
    }
    // neighbours (ascending) into the caller's row, then volume / centroid
    float sx, sy, sz;
    uint32_t alive[kNaPcap / 32];
    const int nv = gather_vertices(c, S, sx, sy, sz, alive);
    int nvals = 0;
#pragma unroll
    for (int w = 0; w < kNaPcap / 32; w++) {
      int f = 32 * w + (int)lane;
      bool isn = ((alive[w] >> lane) & 1u) && S.pid[f] >= 0;
      uint32_t mk = __ballot_sync(FULL, isn);
      if (isn) S.otri[nvals + __popc(mk & lt)] = (uint32_t)S.pid[f];
      nvals += __popc(mk);
    }
    __syncwarp();
    if (nvals > kNaRow) {
      if (lane == 0) overflow_row(i, counts, vol, cen, SC);
      continue;
    }
    int32_t* row = nbrs + (size_t)i * kNaRow;
    for (int t = (int)lane; t < nvals; t += 32) {
      int v = (int)S.otri[t];
      int rank = 0;
      for (int u = 0; u < nvals; u++) rank += (int)S.otri[u] < v;
      row[rank] = v;
    }
    const float cx = sx / nv, cy = sy / nv, cz = sz / nv;
    float V = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f, Sabs = 0.f, emax = 0.f;
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
      float gx = -hgt * pf.x, gy = -hgt * pf.y, gz = -hgt * pf.z;
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
    float L = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) L += fmaxf(c.alo[k] * c.alo[k], c.ahi[k] * c.ahi[k]);
    L = sqrtf(L);
    double ox = cx, oy = cy, oz = cz, Vd = V;
    if (c.fp64 && volume_needs_fp64(V, L, Sabs, emax)) {
      double Mxd, Myd, Mzd;
      volume_fp64(S, nv, c.me, c.box, c.box + 3, sites, (double)cx, (double)cy, (double)cz, Vd, Mxd, Myd, Mzd);
      if (Vd > 0.0) {
        ox += Mxd / Vd;
        oy += Myd / Vd;
        oz += Mzd / Vd;
      }
    } else if (V > 0.0f) {
      ox += Mx / V;
      oy += My / V;
      oz += Mz / V;
    }
    if (lane == 0) {
      counts[i] = nvals;
      vol[i] = (float)Vd;
      cen[3 * (size_t)i] = (float)((double)c.me.x + ox);
      cen[3 * (size_t)i + 1] = (float)((double)c.me.y + oy);
      cen[3 * (size_t)i + 2] = (float)((double)c.me.z + oz);
    }
    __syncwarp();
  }
}

__global__ void na_status_kernel(const NoAllocScratch* S, int32_t* status) { *status = S->error; }

// Device address of the scratch array on the current device. It is looked
// up once per device and CUDA context (with that device current) and cached;
// a cudaDeviceReset gives the device a new context (and the module a new
// copy of the array), so the cache is keyed by the context's id, read through
// two driver calls that the runtime hands out (no link to the driver
// library). If that id cannot be read, the address is looked up on every
// call, which allocates nothing either.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_mu;
struct ScratchSlot {
  void* addr;
  unsigned long long ctx_id;
};
ScratchSlot g_slot[64] = {};
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;
bool g_entry_tried = false;

bool context_id(unsigned long long* id) {
  if (!g_entry_tried) {
    g_entry_tried = true;
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  CUcontext c = nullptr;
  if (!g_get_current || !g_get_id || g_get_current(&c) != CUDA_SUCCESS || !c) return false;
  return g_get_id(c, id) == CUDA_SUCCESS;
}

int scratch_on_device(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  const bool have_id = context_id(&id);
  ScratchSlot& S = g_slot[dev];
  if (!S.addr || !have_id || S.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return VD_ERR_CUDA;
    S.addr = p;
    S.ctx_id = have_id ? id : 0;
  }
  *out = static_cast<NoAllocScratch*>(S.addr);
  return VD_OK;
}

}  // namespace
}  // namespace vd

using namespace vd;

extern "C" int vd_cells_noalloc(const float* sites_xyz, const float* weights, int64_t n, vd_box bbox,
                                int32_t* counts, int32_t* neighbors, float* volume, float* centroid,
                                int32_t* status, void* stream) {
  if (!sites_xyz || !counts || !neighbors || !volume || !centroid || !status || n <= 0) return VD_ERR_INVALID_ARG;
  if (n > kNaMaxSites) return VD_ERR_TOO_LARGE;
  for (int k = 0; k < 3; k++)
    if (!(bbox.lo[k] < bbox.hi[k])) return VD_ERR_INVALID_ARG;
  NoAllocScratch* S = nullptr;
  int rc = scratch_on_device(&S);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the work counter and the error word must start at zero on every call
  if (cudaMemsetAsync(&S->work, 0, 2 * sizeof(int), s) != cudaSuccess) return VD_ERR_CUDA;
  int nn = (int)n;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return VD_ERR_CUDA;
  int blocks = (nn + kNaWarps - 1) / kNaWarps;
  if (sms > 0 && blocks > 4 * sms) blocks = 4 * sms;
  // each launch through cudaLaunchKernel, whose return value is that
  // launch's own status: an error left by the caller's earlier work is
  // neither reported as ours nor cleared
  const float* w = weights;
  void* pack_args[] = {(void*)&sites_xyz, (void*)&w, (void*)&nn, (void*)&bbox, (void*)&S};
  if (cudaLaunchKernel((const void*)na_pack_kernel, dim3((nn + 255) / 256), dim3(256), pack_args, 0, s) !=
      cudaSuccess)
    return VD_ERR_CUDA;
  void* cell_args[] = {(void*)&nn, (void*)&counts, (void*)&neighbors, (void*)&volume, (void*)&centroid, (void*)&S};
  if (cudaLaunchKernel((const void*)na_cells_kernel, dim3(blocks), dim3(32 * kNaWarps), cell_args, 0, s) !=
      cudaSuccess)
    return VD_ERR_CUDA;
  const NoAllocScratch* Sc = S;
  void* st_args[] = {(void*)&Sc, (void*)&status};
  if (cudaLaunchKernel((const void*)na_status_kernel, dim3(1), dim3(1), st_args, 0, s) != cudaSuccess)
    return VD_ERR_CUDA;
  return VD_OK;
}
