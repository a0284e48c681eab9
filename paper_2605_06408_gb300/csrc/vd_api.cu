// vd_api.cu -- the C ABI declared in include/vd.h: context, workspace and
// the order of the kernels of one build (App. A pipeline: pack, BVH,
// fused per-cell kernel; then CSR compaction). Everything is enqueued on
// the caller's stream; nothing here synchronises the host except
// workspace growth (cudaMalloc) and vd_get_status.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <tuple>

#include "vd_big.cuh"

using namespace vd;

namespace {

constexpr int kStride = 64;      // neighbour row stride of the register-resident pass
constexpr int kAmbCap = 1 << 16; // cells recorded with an FP64-ambiguous sign test
constexpr int kHistEntries = 256 * 2 * kSortBlocksMax;

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t off[40];
  int count = 0;
  size_t total = 0;
  size_t add(size_t bytes) {
    size_t o = total;
    off[count++] = o;
    total += align_up(bytes);
    return o;
  }
};

int64_t ovf_capacity(int64_t n) { return n > 4096 ? n : 4096; }
int64_t pool_capacity(int64_t n) { return n > (1 << 22) ? n : (1 << 22); }
int big_warps(int num_sms) { return num_sms * kBigBlocksPerSm * kBigWarpsPerBlock; }

}  // namespace

struct vd_ctx {
  int device = 0;
  int num_sms = 0;
  vd_config cfg;
  // workspace
  char* base = nullptr;
  size_t bytes = 0;
  int64_t cap_n = 0;
  float4* sites = nullptr;
  uint64_t* keys_a = nullptr;
  uint64_t* keys_b = nullptr;
  int* vals_a = nullptr;
  int* vals_b = nullptr;
  int* inv_perm = nullptr;
  unsigned* hist = nullptr;
  int* left = nullptr;
  int* right = nullptr;
  int* parent = nullptr;
  int* visit = nullptr;
  int2* range = nullptr;
  float4* box_lo = nullptr;
  float4* box_hi = nullptr;
  float4* nodes = nullptr;
  int* counts = nullptr;
  int* scratch = nullptr;
  int* pool = nullptr;
  char* arena = nullptr;
  unsigned char* loser = nullptr;
  long long pool_cap = 0;
  int* ovf_list = nullptr;
  int* ovf_slot = nullptr;
  int* blist = nullptr;
  int* vcount = nullptr;  // mesh output: vertices per cell
  int* amb_list = nullptr;  // cells with an FP64-ambiguous sign test (last forward)
  int* knn = nullptr;       // KNN warm start: kKnn nearest sites of every sorted site
  long long* block_sums = nullptr;
  int* work = nullptr;  // [8] work counters
  unsigned* wrange = nullptr;  // [2] orderable min / max weight
  DevStatus* st = nullptr;
  SetInfo* sets_dev = nullptr;
  SetInfo* sets_host = nullptr;  // pinned staging
  int ovf_cap = 0;
  // last forward build
  bool have_forward = false;
  int last_n = 0;
  int last_nsets = 0;
  int set_shift = 63;
  uint64_t* keys_sorted = nullptr;
  int* perm = nullptr;
  cudaStream_t last_stream = nullptr;
  // phase timing (vd_config.timing)
  cudaEvent_t ev[8] = {};
  bool ev_made = false;
  bool ev_valid = false;
  bool ev_backward = false;
  int launches = 0;
  // test hook (environment VD_TEST_STALL_HELPER at vd_create): one helping
  // group of each build's large-cell pass is never counted
  bool test_stall = false;
  // tape of the forward's cells for the adjoint (separate allocation)
  char* tape = nullptr;
  int64_t tape_cap = 0;
  bool tape_valid = false;
  // large-cell tape: polytopes of the cells past the register path
  char* btape = nullptr;
  int64_t btape_cap = 0;
  // autotuner: best configuration per (log2 n, weighted, set count)
  std::map<std::tuple<int, int, int>, vd_config> tuned;
  // partition of the cells (vd_set_partition): this context builds part
  // `part` of `nparts` contiguous ranges of the Morton-sorted order
  int part = 0;
  int nparts = 1;
  int last_begin = 0, last_end = 0;  // the range of the last forward build
};

// events 0..6 bracket the phases: pack | sort | bvh | cells | overflow | csr
static void mark(vd_ctx* ctx, int k, cudaStream_t s) {
  if (!ctx->cfg.timing) return;
  if (!ctx->ev_made) {
    for (int q = 0; q < 8; q++) cudaEventCreate(&ctx->ev[q]);
    ctx->ev_made = true;
  }
  cudaEventRecord(ctx->ev[k], s);
}

static int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return VD_OK;
  return VD_ERR_CUDA;
}

static int check_config(const vd_config* c) {
  if (c->leaf_size < 1 || c->leaf_size > kMaxLeaf) return VD_ERR_INVALID_ARG;
  if (c->verts_per_lane != 2 && c->verts_per_lane != 4) return VD_ERR_INVALID_ARG;
  if (c->queue_per_lane != 1 && c->queue_per_lane != 2 && c->queue_per_lane != 4 && c->queue_per_lane != 8)
    return VD_ERR_INVALID_ARG;
  if (c->cull_mode < 0 || c->cull_mode > 2) return VD_ERR_INVALID_ARG;
  if (c->traversal < 0 || c->traversal > 1) return VD_ERR_INVALID_ARG;
  if (c->warps_per_block < 1 || c->warps_per_block > 8) return VD_ERR_INVALID_ARG;
  if (c->blocks_per_sm < 0 || c->blocks_per_sm > 64) return VD_ERR_INVALID_ARG;
  if (c->counters < 0 || c->counters > 1 || c->timing < 0 || c->timing > 1) return VD_ERR_INVALID_ARG;
  if (c->warm_start < 0 || c->warm_start > 2) return VD_ERR_INVALID_ARG;
  if (c->cell_mode < 0 || c->cell_mode > 1) return VD_ERR_INVALID_ARG;
  if (c->precision < 0 || c->precision > 1) return VD_ERR_INVALID_ARG;
  if (c->tape < 0 || c->tape > 1) return VD_ERR_INVALID_ARG;
  return VD_OK;
}

static int release(vd_ctx* ctx) {
  if (ctx->base) cudaFree(ctx->base);
  ctx->base = nullptr;
  if (ctx->tape) cudaFree(ctx->tape);
  ctx->tape = nullptr;
  ctx->tape_cap = 0;
  ctx->tape_valid = false;
  if (ctx->btape) cudaFree(ctx->btape);
  ctx->btape = nullptr;
  ctx->btape_cap = 0;
  ctx->bytes = 0;
  ctx->cap_n = 0;
  ctx->have_forward = false;
  return VD_OK;
}

static Layout make_layout(int64_t n, int num_sms) {
  Layout L;
  int64_t ovf = ovf_capacity(n);
  int64_t nb = (n + 8191) / 8192 + 1;
  L.add(sizeof(float4) * n);           // 0 sites
  L.add(sizeof(uint64_t) * n);         // 1 keys_a
  L.add(sizeof(uint64_t) * n);         // 2 keys_b
  L.add(sizeof(int) * n);              // 3 vals_a
  L.add(sizeof(int) * n);              // 4 vals_b
  L.add(sizeof(int) * n);              // 5 inv_perm
  L.add(sizeof(unsigned) * kHistEntries);  // 6 hist
  L.add(sizeof(int) * n);              // 7 left
  L.add(sizeof(int) * n);              // 8 right
  L.add(sizeof(int) * 2 * n);          // 9 parent
  L.add(sizeof(int) * n);              // 10 visit
  L.add(sizeof(int2) * n);             // 11 range
  L.add(sizeof(float4) * n);           // 12 box_lo
  L.add(sizeof(float4) * n);           // 13 box_hi
  L.add(sizeof(float4) * 4 * n);       // 14 nodes
  L.add(sizeof(int) * n);              // 15 counts
  L.add(sizeof(int) * (size_t)n * kStride);        // 16 scratch
  L.add(sizeof(int) * (size_t)pool_capacity(n));   // 17 pool
  L.add(sizeof(int) * ovf);            // 18 ovf_list
  L.add(sizeof(int) * n);              // 19 ovf_slot
  L.add(sizeof(int) * ovf);            // 20 blist
  L.add(sizeof(long long) * nb);       // 21 block_sums
  L.add(sizeof(int) * 16);             // 22 work (+ weight range)
  L.add(sizeof(DevStatus));            // 23 status
  L.add(sizeof(SetInfo) * kMaxSets);   // 24 sets
  L.add(big_arena_bytes() * (size_t)big_warps(num_sms));  // 25 arenas
  L.add((size_t)n);                    // 26 duplicate losers
  L.add(sizeof(int) * n);              // 27 mesh vertex count per cell
  L.add(sizeof(int) * kAmbCap);        // 28 cells with an FP64-ambiguous sign test
  L.add(sizeof(int) * kKnn * (size_t)n);  // 29 KNN warm start: nearest sites per site
  return L;
}

// The tape (1 KB per site) when the configuration asks for it and it fits in
// half of the free device memory; otherwise none (the adjoint re-clips).
// Beside it, the large-cell tape (kBigTapePerSite bytes per site, at least
// 64 MB) if that fits in a quarter of what is left; cells whose polytope
// does not fit there are re-clipped by the adjoint.
static void reserve_tape(vd_ctx* ctx) {
  const bool want = ctx->cfg.tape != 0 && ctx->cfg.cell_mode == 0;
  if (!want || ctx->tape_cap >= ctx->cap_n) return;
  if (ctx->tape) cudaFree(ctx->tape);
  ctx->tape = nullptr;
  ctx->tape_cap = 0;
  ctx->tape_valid = false;
  if (ctx->btape) cudaFree(ctx->btape);
  ctx->btape = nullptr;
  ctx->btape_cap = 0;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return;
  const size_t bytes = (size_t)kTapeStride * (size_t)ctx->cap_n;
  if (bytes > free_b / 2) return;
  if (cudaMalloc(&ctx->tape, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->tape = nullptr;
    return;
  }
  ctx->tape_cap = ctx->cap_n;
  const size_t bbytes = std::max((size_t)64 << 20, (size_t)kBigTapePerSite * (size_t)ctx->cap_n);
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && bbytes <= free_b / 4) {
    if (cudaMalloc(&ctx->btape, bbytes) == cudaSuccess) {
      ctx->btape_cap = (int64_t)bbytes;
    } else {
      cudaGetLastError();
      ctx->btape = nullptr;
    }
  }
}

static int reserve(vd_ctx* ctx, int64_t n) {
  if (n <= ctx->cap_n && ctx->base) {
    reserve_tape(ctx);
    return VD_OK;
  }
  int64_t want = n;
  if (ctx->cap_n > 0 && want < ctx->cap_n + ctx->cap_n / 4) want = ctx->cap_n + ctx->cap_n / 4;
  if (want > kMaxSites) want = kMaxSites;
  if (want < 1024) want = 1024;
  Layout L = make_layout(want, ctx->num_sms);
  release(ctx);
  cudaError_t e = cudaMalloc(&ctx->base, L.total);
  if (e != cudaSuccess) {
    ctx->base = nullptr;
    return VD_ERR_CUDA;
  }
  char* b = ctx->base;
  ctx->bytes = L.total;
  ctx->cap_n = want;
  ctx->ovf_cap = (int)ovf_capacity(want);
  ctx->sites = (float4*)(b + L.off[0]);
  ctx->keys_a = (uint64_t*)(b + L.off[1]);
  ctx->keys_b = (uint64_t*)(b + L.off[2]);
  ctx->vals_a = (int*)(b + L.off[3]);
  ctx->vals_b = (int*)(b + L.off[4]);
  ctx->inv_perm = (int*)(b + L.off[5]);
  ctx->hist = (unsigned*)(b + L.off[6]);
  ctx->left = (int*)(b + L.off[7]);
  ctx->right = (int*)(b + L.off[8]);
  ctx->parent = (int*)(b + L.off[9]);
  ctx->visit = (int*)(b + L.off[10]);
  ctx->range = (int2*)(b + L.off[11]);
  ctx->box_lo = (float4*)(b + L.off[12]);
  ctx->box_hi = (float4*)(b + L.off[13]);
  ctx->nodes = (float4*)(b + L.off[14]);
  ctx->counts = (int*)(b + L.off[15]);
  ctx->scratch = (int*)(b + L.off[16]);
  ctx->pool = (int*)(b + L.off[17]);
  ctx->pool_cap = pool_capacity(want);
  ctx->arena = b + L.off[25];
  ctx->loser = (unsigned char*)(b + L.off[26]);
  ctx->vcount = (int*)(b + L.off[27]);
  ctx->amb_list = (int*)(b + L.off[28]);
  ctx->knn = (int*)(b + L.off[29]);
  ctx->ovf_list = (int*)(b + L.off[18]);
  ctx->ovf_slot = (int*)(b + L.off[19]);
  ctx->blist = (int*)(b + L.off[20]);
  ctx->block_sums = (long long*)(b + L.off[21]);
  ctx->work = (int*)(b + L.off[22]);
  ctx->wrange = (unsigned*)(ctx->work + 8);
  ctx->st = (DevStatus*)(b + L.off[23]);
  ctx->sets_dev = (SetInfo*)(b + L.off[24]);
  reserve_tape(ctx);
  return VD_OK;
}

static CellBuffers cell_buffers(vd_ctx* ctx) {
  CellBuffers c;
  std::memset(&c, 0, sizeof(c));
  c.sites = ctx->sites;
  c.loser = ctx->loser;
  c.perm = ctx->perm;
  c.nodes = ctx->nodes;
  c.keys = ctx->keys_sorted;
  c.sets = ctx->sets_dev;
  c.nsets = ctx->last_nsets;
  c.set_shift = ctx->set_shift;
  c.n = ctx->last_n;
  c.counts = ctx->counts;
  c.scratch = ctx->scratch;
  c.stride = kStride;
  c.pool = ctx->pool;
  c.pool_cap = ctx->pool_cap;
  c.arena = ctx->arena;
  c.ovf_list = ctx->ovf_list;
  c.ovf_cap = ctx->ovf_cap;
  c.ovf_slot = ctx->ovf_slot;
  c.work = ctx->work;
  c.st = ctx->st;
  c.cfg = ctx->cfg;
  c.tape = (ctx->cfg.tape && ctx->cfg.cell_mode == 0 && ctx->tape_cap >= ctx->last_n) ? ctx->tape : nullptr;
  c.stall = ctx->test_stall ? ctx->work + 6 : nullptr;
  c.btape = c.tape ? ctx->btape : nullptr;
  c.btape_cap = c.tape ? ctx->btape_cap : 0;
  c.amb_list = ctx->amb_list;
  c.amb_cap = kAmbCap;
  c.cell_begin = ctx->last_begin;
  c.cell_end = ctx->last_end;
  c.knn = ctx->knn;
  return c;
}

static bool box_ok(const vd_box& b) {
  for (int k = 0; k < 3; k++) {
    if (!(b.lo[k] == b.lo[k]) || !(b.hi[k] == b.hi[k])) return false;
    if (!(b.lo[k] < b.hi[k])) return false;
    if (b.lo[k] < -3.0e38f || b.hi[k] > 3.0e38f) return false;
  }
  return true;
}

static bool out_ok(const vd_out* out) {
  if (!out || !out->offsets || !out->nnz_out || !out->volume || !out->centroid) return false;
  if (out->nnz_capacity < 0) return false;
  if (!out->neighbors && out->nnz_capacity > 0) return false;
  return true;
}

// The whole forward pipeline for nsets sets already staged in ctx->sets_host.
static int run_forward(vd_ctx* ctx, const float* xyz, const float* w, int n, int nsets, int set_shift,
                       const vd_out* out, cudaStream_t s) {
  cudaError_t e;
  int rc = reserve(ctx, n);
  if (rc) return rc;
  ctx->have_forward = false;
  ctx->ev_valid = false;
  mark(ctx, 0, s);
  e = cudaMemcpyAsync(ctx->sets_dev, ctx->sets_host, sizeof(SetInfo) * nsets, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s);
  cudaMemsetAsync(ctx->work, 0, sizeof(int) * 8, s);
  if (ctx->test_stall) cudaMemsetAsync(ctx->work + 6, 1, sizeof(int), s);  // arm the test hook's token
  cudaMemsetAsync(ctx->ovf_slot, 0xff, sizeof(int) * (size_t)n, s);
  cudaMemsetAsync(ctx->counts, 0, sizeof(int) * (size_t)n, s);
  // 1. keys: (set, weight stratum, Morton code in the set's box); input validation
  e = launch_weight_range(w, n, ctx->sets_dev, nsets, ctx->wrange, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  const int bin_shift = nsets > 1 ? 51 : 60;
  e = launch_pack_keys(xyz, w, n, ctx->sets_dev, nsets, set_shift, bin_shift, ctx->wrange, ctx->keys_a,
                       ctx->vals_a, ctx->st, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  mark(ctx, 1, s);
  // 2. radix sort of (key, index)
  uint64_t* k0 = ctx->keys_a;
  uint64_t* k1 = ctx->keys_b;
  int* v0 = ctx->vals_a;
  int* v1 = ctx->vals_b;
  int bits = nsets > 1 ? 64 : 63;
  e = radix_sort_pairs(k0, k1, v0, v1, ctx->hist, n, bits, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  ctx->keys_sorted = k0;
  ctx->perm = v0;
  mark(ctx, 2, s);
  // 3. packed float4 sites in Morton order (App. A.1)
  e = launch_gather_sites(xyz, w, ctx->perm, n, ctx->sets_dev, ctx->keys_sorted, set_shift, nsets, ctx->sites, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  e = launch_inverse_perm(ctx->perm, n, ctx->inv_perm, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  e = launch_mark_losers(ctx->keys_sorted, ctx->sites, ctx->perm, n, ctx->loser, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  // 4. LBVH with per-node max weight (App. A.2)
  BvhBuffers b;
  b.keys = ctx->keys_sorted;
  b.keys_alt = nullptr;
  b.vals = nullptr;
  b.vals_alt = nullptr;
  b.hist = nullptr;
  b.left = ctx->left;
  b.right = ctx->right;
  b.parent = ctx->parent;
  b.range = ctx->range;
  b.visit = ctx->visit;
  b.box_lo = ctx->box_lo;
  b.box_hi = ctx->box_hi;
  b.nodes = ctx->nodes;
  e = launch_build_bvh(ctx->keys_sorted, ctx->sites, n, ctx->cfg.leaf_size, b, ctx->sets_dev, nsets, ctx->st, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  // 5. fused traversal + cull + clip (Alg. 1, Sec. 4, App. B), over this
  // context's part of the sorted order; the other cells get no neighbours
  // and volume / centroid 0
  ctx->last_n = n;
  ctx->last_nsets = nsets;
  ctx->set_shift = set_shift;
  ctx->last_begin = (int)(((int64_t)n * ctx->part) / ctx->nparts);
  ctx->last_end = (int)(((int64_t)n * (ctx->part + 1)) / ctx->nparts);
  if (ctx->nparts > 1) {
    cudaMemsetAsync(out->volume, 0, sizeof(float) * (size_t)n, s);
    cudaMemsetAsync(out->centroid, 0, sizeof(float) * 3 * (size_t)n, s);
  }
  CellBuffers c = cell_buffers(ctx);
  c.vol = out->volume;
  c.cen = out->centroid;
  const bool knn = ctx->cfg.warm_start == 2 && ctx->cfg.cell_mode == 0;
  if (knn) {  // the KNN warm start's lists (App. A.6), for this build's cells
    e = launch_knn(c, ctx->knn, s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
  }
  mark(ctx, 3, s);
  e = launch_cells(c, ctx->num_sms, s, [&]() { mark(ctx, 4, s); });
  if (e != cudaSuccess) return VD_ERR_CUDA;
  mark(ctx, 5, s);
  // 6. CSR
  e = launch_csr(c, out->offsets, out->neighbors, out->nnz_capacity, out->nnz_out, ctx->block_sums, out->status,
                 true, s);
  if (e != cudaSuccess) return VD_ERR_CUDA;
  mark(ctx, 6, s);
  ctx->have_forward = true;
  ctx->tape_valid = c.tape != nullptr;
  ctx->last_stream = s;
  ctx->ev_valid = ctx->cfg.timing != 0;
  ctx->ev_backward = false;
  int passes = (bits + 7) / 8;
  ctx->launches = (w ? 1 : 0) + 1 + 3 * passes + 3 + (n >= 2 ? 4 : 1) + 2 + 3 +
                  (out->neighbors && out->nnz_capacity > 0) + 1 + (knn ? 1 : 0);
  return VD_OK;
}

extern "C" {

int vd_default_config(vd_config* cfg) {
  if (!cfg) return VD_ERR_INVALID_ARG;
  cfg->leaf_size = 16;
  cfg->verts_per_lane = 2;
  cfg->queue_per_lane = 4;
  cfg->cull_mode = 0;
  cfg->traversal = 0;
  cfg->warps_per_block = 4;
  cfg->blocks_per_sm = 0;
  cfg->counters = 0;
  cfg->timing = 0;
  cfg->warm_start = 0;
  cfg->cell_mode = 0;
  cfg->tape = 0;
  cfg->precision = 0;
  return VD_OK;
}

int vd_create(vd_ctx** out, int device, const vd_config* cfg) {
  if (!out) return VD_ERR_INVALID_ARG;
  *out = nullptr;
  vd_config c;
  vd_default_config(&c);
  if (cfg) {
    c = *cfg;
    int rc = check_config(&c);
    if (rc) return rc;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VD_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return VD_ERR_CUDA;
  vd_ctx* ctx = new (std::nothrow) vd_ctx();
  if (!ctx) return VD_ERR_CUDA;
  ctx->device = device;
  ctx->cfg = c;
  ctx->test_stall = std::getenv("VD_TEST_STALL_HELPER") != nullptr;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    return VD_ERR_CUDA;
  }
  if (cudaMallocHost(&ctx->sets_host, sizeof(SetInfo) * kMaxSets) != cudaSuccess) {
    delete ctx;
    return VD_ERR_CUDA;
  }
  *out = ctx;
  return VD_OK;
}

int vd_destroy(vd_ctx* ctx) {
  if (!ctx) return VD_OK;
  cudaSetDevice(ctx->device);
  release(ctx);
  if (ctx->sets_host) cudaFreeHost(ctx->sets_host);
  if (ctx->ev_made)
    for (int q = 0; q < 8; q++) cudaEventDestroy(ctx->ev[q]);
  delete ctx;
  return VD_OK;
}

int vd_set_config(vd_ctx* ctx, const vd_config* cfg) {
  if (!ctx || !cfg) return VD_ERR_INVALID_ARG;
  int rc = check_config(cfg);
  if (rc) return rc;
  ctx->cfg = *cfg;
  return VD_OK;
}

int vd_set_partition(vd_ctx* ctx, int32_t part, int32_t nparts) {
  if (!ctx || nparts < 1 || part < 0 || part >= nparts) return VD_ERR_INVALID_ARG;
  ctx->part = part;
  ctx->nparts = nparts;
  return VD_OK;
}

int vd_reserve(vd_ctx* ctx, int64_t n, int /*weighted*/) {
  if (!ctx || n <= 0) return VD_ERR_INVALID_ARG;
  if (n > kMaxSites) return VD_ERR_TOO_LARGE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  return reserve(ctx, n);
}

size_t vd_workspace_bytes(int64_t n, int /*weighted*/) {
  if (n <= 0) return 0;
  if (n < 1024) n = 1024;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) sms = v;
  } else {
    cudaGetLastError();
  }
  return make_layout(n, sms).total;
}

int vd_build(vd_ctx* ctx, const float* xyz, const float* weights, int64_t n, vd_box bbox, const vd_out* out,
             void* stream) {
  if (!ctx || !xyz || n <= 0 || !box_ok(bbox) || !out_ok(out)) return VD_ERR_INVALID_ARG;
  if (n > kMaxSites) return VD_ERR_TOO_LARGE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  SetInfo& S = ctx->sets_host[0];
  for (int k = 0; k < 3; k++) {
    S.lo[k] = bbox.lo[k];
    S.hi[k] = bbox.hi[k];
  }
  S.first = 0;
  S.count = (int)n;
  S.root = 0;
  S.weighted = weights ? 1 : 0;
  return run_forward(ctx, xyz, weights, (int)n, 1, 63, out, (cudaStream_t)stream);
}

int vd_copy_neighbors(vd_ctx* ctx, const vd_out* out, void* stream) {
  if (!ctx || !out || !out->offsets || !out->nnz_out || out->nnz_capacity < 0) return VD_ERR_INVALID_ARG;
  if (!ctx->have_forward) return VD_ERR_NO_FORWARD;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  CellBuffers c = cell_buffers(ctx);
  // clear a previous capacity error, keep any other
  cudaError_t e = launch_csr(c, out->offsets, out->neighbors, out->nnz_capacity, out->nnz_out, ctx->block_sums,
                             out->status, true, s);
  ctx->last_stream = s;
  return cuda_fail(e);
}

int vd_build_batched(vd_ctx* ctx, const float* xyz, const float* weights, const int64_t* set_offsets,
                     const vd_box* boxes, const uint8_t* weighted, int32_t nsets, const vd_out* out, void* stream) {
  if (!ctx || !xyz || !set_offsets || !boxes || nsets < 1 || nsets > kMaxSets || !out_ok(out))
    return VD_ERR_INVALID_ARG;
  if (set_offsets[0] != 0) return VD_ERR_INVALID_ARG;
  for (int s = 0; s < nsets; s++) {
    if (set_offsets[s + 1] < set_offsets[s]) return VD_ERR_INVALID_ARG;
    if (!box_ok(boxes[s])) return VD_ERR_INVALID_ARG;
  }
  int64_t n = set_offsets[nsets];
  if (n <= 0) return VD_ERR_INVALID_ARG;
  if (n > kMaxSites) return VD_ERR_TOO_LARGE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  for (int s = 0; s < nsets; s++) {
    SetInfo& S = ctx->sets_host[s];
    for (int k = 0; k < 3; k++) {
      S.lo[k] = boxes[s].lo[k];
      S.hi[k] = boxes[s].hi[k];
    }
    S.first = (int)set_offsets[s];
    S.count = (int)(set_offsets[s + 1] - set_offsets[s]);
    S.root = 0;
    S.weighted = weights ? (weighted ? (weighted[s] ? 1 : 0) : 1) : 0;
  }
  // 10-bit set id, 3-bit weight stratum, 17-bit Morton coordinates
  return run_forward(ctx, xyz, weights, (int)n, nsets, 54, out, (cudaStream_t)stream);
}

}  // extern "C"

// One pass of the adjoint kernels over the last build's cells: gradients
// (mode 0), mesh vertex counts (1) or mesh output (2).
static int back_pass(vd_ctx* ctx, BackBuffers b, cudaStream_t s) {
  cudaMemsetAsync(ctx->work + 2, 0, sizeof(int) * 3, s);
  b.c = cell_buffers(ctx);
  b.inv_perm = ctx->inv_perm;
  b.list = ctx->blist;
  b.list_count = ctx->work + 4;
  b.list_cap = ctx->ovf_cap;
  b.work = ctx->work + 2;
  return cuda_fail(launch_backward(b, ctx->num_sms, s));
}

static int backward_common(vd_ctx* ctx, const float* grad_volume, const float* grad_centroid,
                           const float* grad_vertices, const int32_t* vertex_offsets, float* grad_sites,
                           float* grad_weights, int recompute, cudaStream_t s) {
  int n = ctx->last_n;
  cudaMemsetAsync(grad_sites, 0, sizeof(float) * 3 * (size_t)n, s);
  if (grad_weights) cudaMemsetAsync(grad_weights, 0, sizeof(float) * (size_t)n, s);
  cudaMemsetAsync(&ctx->st->error, 0, sizeof(int), s);
  cudaMemsetAsync(&ctx->st->btape_restored, 0, sizeof(long long), s);
  BackBuffers b;
  std::memset(&b, 0, sizeof(b));
  b.gvol = grad_volume;
  b.gcen = grad_centroid;
  b.gp = grad_sites;
  b.gw = grad_weights;
  b.tape = (recompute == 0 && ctx->tape_valid) ? ctx->tape : nullptr;
  b.mode = 0;
  b.gvert = grad_vertices;
  b.voff = vertex_offsets;
  ctx->ev_valid = false;
  mark(ctx, 0, s);
  int rc = back_pass(ctx, b, s);
  mark(ctx, 6, s);
  ctx->last_stream = s;
  ctx->ev_valid = ctx->cfg.timing != 0;
  ctx->ev_backward = true;
  ctx->launches = 2;
  return rc;
}

extern "C" {

int vd_backward(vd_ctx* ctx, const float* grad_volume, const float* grad_centroid, float* grad_sites,
                float* grad_weights, int recompute, void* stream) {
  if (!ctx || !grad_sites || (recompute != 0 && recompute != 1)) return VD_ERR_INVALID_ARG;
  if (!ctx->have_forward) return VD_ERR_NO_FORWARD;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  return backward_common(ctx, grad_volume, grad_centroid, nullptr, nullptr, grad_sites, grad_weights, recompute,
                         (cudaStream_t)stream);
}

int vd_cells_mesh(vd_ctx* ctx, const vd_mesh* out, void* stream) {
  if (!ctx || !out || !out->vertex_offsets || !out->nverts_out || out->capacity < 0) return VD_ERR_INVALID_ARG;
  if (out->capacity > 0 && (!out->vertices || !out->vertex_sites)) return VD_ERR_INVALID_ARG;
  if (!ctx->have_forward) return VD_ERR_NO_FORWARD;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = ctx->last_n;
  cudaMemsetAsync(&ctx->st->error, 0, sizeof(int), s);
  cudaMemsetAsync(ctx->vcount, 0, sizeof(int) * (size_t)n, s);
  BackBuffers b;
  std::memset(&b, 0, sizeof(b));
  b.tape = ctx->tape_valid ? ctx->tape : nullptr;  // the cells vd_backward(recompute = 0) uses
  b.mode = 1;
  b.vcount = ctx->vcount;
  int rc = back_pass(ctx, b, s);
  if (rc) return rc;
  if (launch_scan(ctx->vcount, n, out->vertex_offsets, ctx->block_sums, &ctx->st->nverts, ctx->st, s) !=
      cudaSuccess)
    return VD_ERR_CUDA;
  if (out->capacity > 0) {
    b.mode = 2;
    b.voff = out->vertex_offsets;
    b.vout = out->vertices;
    b.vsites = out->vertex_sites;
    b.vcap = out->capacity;
    rc = back_pass(ctx, b, s);
    if (rc) return rc;
  }
  ctx->last_stream = s;
  return cuda_fail(launch_mesh_finish(ctx->st, out->nverts_out, out->status, s));
}

int vd_backward_mesh(vd_ctx* ctx, const float* grad_volume, const float* grad_centroid, const float* grad_vertices,
                     const int32_t* vertex_offsets, float* grad_sites, float* grad_weights, void* stream) {
  if (!ctx || !grad_sites || (grad_vertices && !vertex_offsets)) return VD_ERR_INVALID_ARG;
  if (!ctx->have_forward) return VD_ERR_NO_FORWARD;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  return backward_common(ctx, grad_volume, grad_centroid, grad_vertices, vertex_offsets, grad_sites, grad_weights,
                         0, (cudaStream_t)stream);
}

int vd_get_timings(vd_ctx* ctx, vd_timings* t) {
  if (!ctx || !t) return VD_ERR_INVALID_ARG;
  std::memset(t, 0, sizeof(*t));
  t->launches = ctx->launches;
  if (!ctx->ev_valid) return VD_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return VD_ERR_CUDA;
  auto el = [&](int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]);
    return ms;
  };
  if (ctx->ev_backward) {
    t->backward_ms = el(0, 6);
    t->total_ms = t->backward_ms;
  } else {
    t->pack_ms = el(0, 1);
    t->sort_ms = el(1, 2);
    t->bvh_ms = el(2, 3);
    t->cells_ms = el(3, 4);
    t->overflow_ms = el(4, 5);
    t->csr_ms = el(5, 6);
    t->total_ms = el(0, 6);
  }
  return VD_OK;
}

int vd_get_status(vd_ctx* ctx, vd_status* st) {
  if (!ctx || !st) return VD_ERR_INVALID_ARG;
  std::memset(st, 0, sizeof(*st));
  if (!ctx->st) return VD_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return VD_ERR_CUDA;
  DevStatus d;
  if (cudaMemcpy(&d, ctx->st, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess) return VD_ERR_CUDA;
  st->error = d.error;
  st->nnz = d.nnz;
  st->empty_cells = d.empty_cells;
  st->overflow_cells = d.overflow_cells;
  st->failed_cells = d.failed_cells;
  st->fp64_fallbacks = d.fp64_fallbacks;
  st->fp64_ambiguous = d.fp64_ambiguous;
  st->candidates = d.candidates;
  st->clips = d.clips;
  st->nodes = d.nodes;
  st->vertex_tests = d.vertex_tests;
  st->new_vertices = d.new_vertices;
  st->refined_vertices = d.refined_vertices;
  st->refined_volumes = d.refined_volumes;
  for (int k = 0; k < 4; k++) st->overflow_reason[k] = d.ovf_reason[k];
  st->large_candidates = d.large_candidates;
  st->large_clips = d.large_clips;
  st->large_nodes = d.large_nodes;
  st->large_vertex_tests = d.large_vtests;
  st->large_new_vertices = d.large_newv;
  st->large_tape_records = d.btape_records;
  st->large_tape_restored = d.btape_restored;
  st->ambiguous_cells = d.amb_count;
  return VD_OK;
}

int vd_ambiguous_cells(vd_ctx* ctx, int64_t* cells, int64_t capacity, int64_t* count) {
  if (!ctx || !count || capacity < 0 || (capacity > 0 && !cells)) return VD_ERR_INVALID_ARG;
  *count = 0;
  if (!ctx->st || !ctx->have_forward) return VD_ERR_NO_FORWARD;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return VD_ERR_CUDA;
  int total = 0;
  if (cudaMemcpy(&total, &ctx->st->amb_count, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VD_ERR_CUDA;
  *count = total;
  const int64_t m = std::min<int64_t>(std::min<int64_t>(total, kAmbCap), capacity);
  if (m <= 0) return VD_OK;
  int* tmp = new (std::nothrow) int[m];
  if (!tmp) return VD_ERR_CUDA;
  cudaError_t e = cudaMemcpy(tmp, ctx->amb_list, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost);
  for (int64_t k = 0; k < m; k++) cells[k] = tmp[k];
  delete[] tmp;
  return e == cudaSuccess ? VD_OK : VD_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner
//
// Coordinate descent over the kernel form and its capacities: starting from
// the context's configuration, each knob in turn (cell form, warm start,
// polytope capacity, queue depth, leaf size, block size) takes each of
// its other values; a trial is one warm-up build then the faster of two
// timed builds (CUDA events on the caller's stream) of the caller's input,
// and a value is kept if it is at least 2% faster. A configuration under
// which a cell fails (error other than neighbour capacity) is skipped.
static int autotune(vd_ctx* ctx, int64_t n, int nsets, int weighted, const std::function<int(const vd_out*)>& build,
                    int32_t max_trials, int32_t flags, vd_config* best, cudaStream_t s) {
  const vd_config user = ctx->cfg;
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= n) lg++;
  const auto key = std::make_tuple(lg, weighted, nsets > 1 ? 1 + (nsets > 64) : 0);
  if (!(flags & VD_TUNE_FORCE)) {
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
      vd_config c = it->second;
      c.counters = user.counters;
      c.timing = user.timing;
      c.cull_mode = user.cull_mode;
      c.traversal = user.traversal;
      c.precision = user.precision;
      c.tape = user.tape;
      ctx->cfg = c;
      if (best) *best = c;
      return VD_OK;
    }
  }
  if (max_trials <= 0) max_trials = 16;
  // scratch outputs of the trial builds
  const int64_t cap = 24 * n + 4096;
  vd_out o{};
  char* mem = nullptr;
  const size_t b_off = align_up(sizeof(int32_t) * (size_t)(n + 1)), b_nb = align_up(sizeof(int32_t) * (size_t)cap),
               b_vol = align_up(sizeof(float) * (size_t)n), b_cen = align_up(sizeof(float) * 3 * (size_t)n);
  if (cudaMalloc(&mem, b_off + b_nb + b_vol + b_cen + 512) != cudaSuccess) return VD_ERR_CUDA;
  o.offsets = (int32_t*)mem;
  o.neighbors = (int32_t*)(mem + b_off);
  o.nnz_capacity = cap;
  o.volume = (float*)(mem + b_off + b_nb);
  o.centroid = (float*)(mem + b_off + b_nb + b_vol);
  o.nnz_out = (int64_t*)(mem + b_off + b_nb + b_vol + b_cen);
  o.status = (int32_t*)(mem + b_off + b_nb + b_vol + b_cen + 256);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int trials = 0;
  auto trial = [&](vd_config c, float& ms) -> bool {
    c.counters = 0;
    c.timing = 0;
    if (check_config(&c) != VD_OK) return false;
    ctx->cfg = c;
    trials++;
    if (build(&o) != VD_OK) return false;
    vd_status st;
    if (vd_get_status(ctx, &st) != VD_OK) return false;
    if (st.error != VD_OK && st.error != VD_ERR_CAPACITY) return false;
    ms = INFINITY;
    for (int r = 0; r < 2; r++) {
      cudaEventRecord(e0, s);
      if (build(&o) != VD_OK) return false;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return false;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms = fminf(ms, t);
    }
    return true;
  };
  vd_config cur = user;
  float cur_ms = INFINITY;
  int rc = VD_OK;
  if (!trial(cur, cur_ms)) {
    // the starting point itself failed: fall back to the defaults
    vd_default_config(&cur);
    cur.cull_mode = user.cull_mode;
    cur.traversal = user.traversal;
    cur.precision = user.precision;
    if (!trial(cur, cur_ms)) rc = VD_ERR_CELL_OVERFLOW;
  }
  if (rc == VD_OK) {
    struct Knob {
      int32_t vd_config::*field;
      int values[3];
      int count;
      bool warp_only;
    };
    // the warm start comes before the leaf size: the best leaf size depends
    // on it (with the KNN start, larger leaves win on every workload here)
    const Knob knobs[] = {
        {&vd_config::cell_mode, {0, 1, 0}, 2, false},     {&vd_config::warm_start, {0, 1, 2}, 3, true},
        {&vd_config::verts_per_lane, {2, 4, 0}, 2, true}, {&vd_config::queue_per_lane, {2, 4, 8}, 3, true},
        {&vd_config::leaf_size, {8, 16, 32}, 3, false},   {&vd_config::warps_per_block, {2, 4, 8}, 3, true},
    };
    for (const Knob& k : knobs) {
      if (k.warp_only && cur.cell_mode != 0) continue;
      for (int v = 0; v < k.count && trials < max_trials; v++) {
        if (cur.*(k.field) == k.values[v]) continue;
        vd_config c = cur;
        c.*(k.field) = k.values[v];
        float ms = INFINITY;
        if (trial(c, ms) && ms < 0.98f * cur_ms) {
          cur = c;
          cur_ms = ms;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(mem);
  // the trial builds' outputs are gone: no forward state for vd_backward
  ctx->have_forward = false;
  cur.counters = user.counters;
  cur.timing = user.timing;
  if (rc != VD_OK) {
    ctx->cfg = user;
    return rc;
  }
  ctx->cfg = cur;
  ctx->tuned[key] = cur;
  if (best) *best = cur;
  return VD_OK;
}

extern "C" {

int vd_autotune(vd_ctx* ctx, const float* xyz, const float* weights, int64_t n, vd_box bbox, int32_t max_trials,
                int32_t flags, vd_config* best, void* stream) {
  if (!ctx || !xyz || n <= 0 || !box_ok(bbox)) return VD_ERR_INVALID_ARG;
  if (n > kMaxSites) return VD_ERR_TOO_LARGE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  return autotune(
      ctx, n, 1, weights ? 1 : 0, [&](const vd_out* o) { return vd_build(ctx, xyz, weights, n, bbox, o, stream); },
      max_trials, flags, best, s);
}

int vd_autotune_batched(vd_ctx* ctx, const float* xyz, const float* weights, const int64_t* set_offsets,
                        const vd_box* boxes, const uint8_t* weighted, int32_t nsets, int32_t max_trials, int32_t flags,
                        vd_config* best, void* stream) {
  if (!ctx || !xyz || !set_offsets || !boxes || nsets < 1 || nsets > kMaxSets) return VD_ERR_INVALID_ARG;
  const int64_t n = set_offsets[nsets];
  if (n <= 0) return VD_ERR_INVALID_ARG;
  if (n > kMaxSites) return VD_ERR_TOO_LARGE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return VD_ERR_CUDA;
  int anyw = 0;
  for (int k = 0; weights && weighted && k < nsets; k++) anyw |= weighted[k] ? 1 : 0;
  return autotune(
      ctx, n, nsets, anyw,
      [&](const vd_out* o) {
        return vd_build_batched(ctx, xyz, weights, set_offsets, boxes, weighted, nsets, o, stream);
      },
      max_trials, flags, best, (cudaStream_t)stream);
}

const char* vd_error_string(int code) {
  switch (code) {
    case VD_OK:
      return "ok";
    case VD_ERR_INVALID_ARG:
      return "invalid argument (n, pointers, box, or a non-finite coordinate or weight)";
    case VD_ERR_CUDA:
      return "CUDA call failed";
    case VD_ERR_CAPACITY:
      return "neighbour capacity too small; *nnz_out holds the required size";
    case VD_ERR_CELL_OVERFLOW:
      return "a cell exceeded the largest polytope capacity";
    case VD_ERR_NO_FORWARD:
      return "no forward build in this context";
    case VD_ERR_TOO_LARGE:
      return "too many sites or neighbours for the index encoding";
    case VD_ERR_TIMEOUT:
      return "a bounded wait between warps of a block ran out (build not valid)";
    default:
      return "unknown error";
  }
}

}  // extern "C"
