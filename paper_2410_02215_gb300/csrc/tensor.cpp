// Context, tensor objects (packed sector table), allocation and error handling.
#include <algorithm>
#include <cstring>
#include <cstdio>
#include <mutex>

#include "common.h"

namespace ftn {

static thread_local std::string g_last_error = "no error";

ftn_status set_error(ftn_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

ftn_status cuda_error(cudaError_t e, const char* where) {
  return set_error(FTN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t dtype_size(ftn_dtype d) { return d == FTN_F64 ? 8 : 4; }

// Device memory of a context without a caller allocator: blocks from the
// stream-ordered allocator on the context's stream, rounded to a size class
// (256-byte steps up to 4 KB, then four classes per power of two) and, once
// freed, kept for the context's later allocations of the same class.  All of
// a context's work is ordered on its stream, so a block freed after the
// launches that use it and handed out again to launches enqueued later is
// never used by both at once (the guarantee cudaFreeAsync and
// cudaMallocAsync give on one stream); the driver's allocator, whose calls
// serialise when several host threads drive contexts, is left out of the
// steady state.  Cached free blocks beyond CACHE_LIMIT go back to it.
// While the stream is being captured into a CUDA graph the cache is not
// used at all: a block allocated in the capture belongs to the graph, and a
// block the graph refers to must never be handed out again.
namespace {
constexpr size_t CACHE_LIMIT = (size_t)2 << 30;

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    (void)cudaGetLastError();
    return true;  // cannot tell (legacy stream beside a capture): the safe answer
  }
  return st != cudaStreamCaptureStatusNone;
}

size_t size_class(size_t b) {
  if (b <= 4096) return (b + 255) & ~(size_t)255;
  int e = 63;
  while (!((b - 1) >> e)) --e;  // 2^e <= b - 1 < 2^(e + 1)
  const size_t step = (size_t)1 << (e - 2);
  return (b + step - 1) & ~(step - 1);
}
}  // namespace

void* dev_alloc(ftn_ctx ctx, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (ctx->alloc) return ctx->alloc(bytes, ctx->user);
  if (capturing(ctx->stream)) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) return nullptr;
    return p;
  }
  const size_t cls = size_class(bytes);
  {
    std::lock_guard<std::mutex> lock(ctx->cache_mu);
    auto it = ctx->free_blocks.find(cls);
    if (it != ctx->free_blocks.end() && !it->second.empty()) {
      void* p = it->second.back();
      it->second.pop_back();
      ctx->cached_bytes -= cls;
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocAsync(&p, cls, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    release_cached_blocks(ctx);  // one retry with the cache handed back
    if (cudaMallocAsync(&p, cls, ctx->stream) != cudaSuccess) return nullptr;
  }
  std::lock_guard<std::mutex> lock(ctx->cache_mu);
  ctx->block_class[p] = cls;
  return p;
}

void dev_free(ftn_ctx ctx, void* p) {
  if (!p) return;
  if (ctx->free_fn) {
    ctx->free_fn(p, ctx->user);
    return;
  }
  const bool cap = capturing(ctx->stream);
  std::unique_lock<std::mutex> lock(ctx->cache_mu);
  auto it = ctx->block_class.find(p);
  if (it == ctx->block_class.end()) {  // allocated during a capture: a plain stream-ordered free
    lock.unlock();
    cudaFreeAsync(p, ctx->stream);
    return;
  }
  const size_t cls = it->second;
  if (cap || ctx->cached_bytes + cls > CACHE_LIMIT) {
    ctx->block_class.erase(it);
    lock.unlock();
    cudaFreeAsync(p, ctx->stream);
    return;
  }
  ctx->free_blocks[cls].push_back(p);
  ctx->cached_bytes += cls;
}

void release_cached_blocks(ftn_ctx ctx) {
  std::lock_guard<std::mutex> lock(ctx->cache_mu);
  for (auto& kv : ctx->free_blocks)
    for (void* p : kv.second) {
      ctx->block_class.erase(p);
      cudaFreeAsync(p, ctx->stream);
    }
  ctx->free_blocks.clear();
  ctx->cached_bytes = 0;
}

void* workspace(ftn_ctx ctx, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes <= ctx->ws_bytes) return ctx->ws;
  dev_free(ctx, ctx->ws);
  size_t want = std::max(bytes, ctx->ws_bytes + ctx->ws_bytes / 2);
  ctx->ws = dev_alloc(ctx, want);
  ctx->ws_bytes = ctx->ws ? want : 0;
  return ctx->ws;
}

int64_t block_size(const ftn_tensor_s* t, uint32_t mask) {
  int64_t s = 1;
  for (int k = 0; k < t->rank; ++k) s *= leg_dim(t, k, mask);
  return s;
}

static ftn_status fill_meta(ftn_tensor_s* t, int rank, const int32_t* d0, const int32_t* d1, const uint8_t* dual,
                            int parity, ftn_dtype dtype) {
  if (rank < 0 || rank > FTN_MAX_RANK) return set_error(FTN_EINVAL, "rank out of range");
  if (parity != 0 && parity != 1) return set_error(FTN_EPARITY, "parity must be 0 or 1");
  if (dtype != FTN_F64 && dtype != FTN_F32) return set_error(FTN_EINVAL, "bad dtype");
  if (rank > 0 && (!d0 || !d1 || !dual)) return set_error(FTN_EINVAL, "null leg arrays");
  t->rank = rank;
  t->parity = parity;
  t->dtype = dtype;
  for (int k = 0; k < rank; ++k) {
    if (d0[k] < 0 || d1[k] < 0) return set_error(FTN_EINVAL, "negative sector dimension");
    if (dual[k] > 1) return set_error(FTN_EINVAL, "dual must be 0 or 1");
    t->d0[k] = d0[k];
    t->d1[k] = d1[k];
    t->dual[k] = dual[k];
  }
  int64_t nb = nblocks(rank, parity);
  t->offsets.resize(nb);
  int64_t off = 0;
  for (int64_t b = 0; b < nb; ++b) {
    t->offsets[b] = off;
    off += block_size(t, block_mask(rank, parity, b));
  }
  t->numel = off;
  return FTN_OK;
}

bool same_meta(const ftn_tensor_s* a, int rank, const int32_t* d0, const int32_t* d1, const uint8_t* dual,
               int parity, ftn_dtype dtype) {
  if (a->rank != rank || a->parity != parity || a->dtype != dtype) return false;
  for (int k = 0; k < rank; ++k)
    if (a->d0[k] != d0[k] || a->d1[k] != d1[k] || a->dual[k] != dual[k]) return false;
  return true;
}

ftn_status make_tensor(ftn_ctx ctx, int rank, const int32_t* d0, const int32_t* d1, const uint8_t* dual,
                       int parity, ftn_dtype dtype, ftn_tensor* out) {
  if (!ctx || !out) return set_error(FTN_EINVAL, "null argument");
  auto* t = new ftn_tensor_s();
  t->ctx = ctx;
  ftn_status st = fill_meta(t, rank, d0, d1, dual, parity, dtype);
  if (st != FTN_OK) {
    delete t;
    return st;
  }
  t->data = dev_alloc(ctx, (size_t)t->numel * dtype_size(dtype));
  if (!t->data) {
    delete t;
    return set_error(FTN_ENOMEM, "device allocation failed");
  }
  t->owned = true;
  *out = t;
  return FTN_OK;
}

bool stream_capturing(cudaStream_t s) { return capturing(s); }

const void* capture_source(ftn_ctx ctx, const void* host, size_t bytes) {
  if (!bytes || !capturing(ctx->stream)) return host;
  // a pinned allocation is not a stream operation: allowed on this thread
  // for the duration of the call in relaxed capture mode
  cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  cudaThreadExchangeStreamCaptureMode(&mode);
  void* p = nullptr;
  const cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocDefault);
  cudaThreadExchangeStreamCaptureMode(&mode);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  std::memcpy(p, host, bytes);
  ctx->graph_host.push_back(p);
  return p;
}

ftn_status upload_table(ftn_ctx ctx, const void* host, size_t bytes, void** dev) {
  *dev = dev_alloc(ctx, bytes);
  if (!*dev) return set_error(FTN_ENOMEM, "device allocation failed (table)");
  const void* src = capture_source(ctx, host, bytes);
  if (!src) return set_error(FTN_ENOMEM, "pinned host allocation failed (table under stream capture)");
  if (bytes) FTN_CUDA(cudaMemcpyAsync(*dev, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return FTN_OK;
}

// ---- table staging ----------------------------------------------------------------
// A small copy from pageable memory is staged by the driver when the call
// returns, so the buffer is free for the next table at once.  (Measured: a
// pinned ring with asynchronous copies was slower with several contexts on
// their own streams.)
void* staging_begin(ftn_ctx ctx, size_t bytes) {
  ctx->stage.resize(std::max<size_t>(bytes, 256));
  return ctx->stage.data();
}

ftn_status staging_upload(ftn_ctx ctx, size_t bytes, void** dev) {
  return upload_table(ctx, ctx->stage.data(), bytes, dev);
}

// ---- permute job builder ------------------------------------------------------
void add_perm_job(std::vector<PermJob>& jobs, int64_t& tiles, int rank, const int64_t* dims_in,
                  const int64_t* dstr_in, int64_t src_off, int64_t dst_off, int sign) {
  // drop unit legs and merge neighbours contiguous in both layouts
  int64_t dims[MAXR], dstr[MAXR];
  int r = 0;
  int64_t total = 1;
  for (int k = 0; k < rank; ++k) {
    total *= dims_in[k];
    if (dims_in[k] == 1) continue;
    if (r > 0 && dstr[r - 1] == dstr_in[k] * dims_in[k]) {
      dims[r - 1] *= dims_in[k];
      dstr[r - 1] = dstr_in[k];
      continue;
    }
    dims[r] = dims_in[k];
    dstr[r] = dstr_in[k];
    ++r;
  }
  if (total == 0) return;
  if (r == 0) {
    dims[0] = 1;
    dstr[0] = 1;
    r = 1;
  }
  int64_t sstr[MAXR];
  int64_t s = 1;
  for (int k = r - 1; k >= 0; --k) {
    sstr[k] = s;
    s *= dims[k];
  }
  // Tile groups.  I: a suffix of the source, read as contiguous rows (the
  // tile's columns); O: legs by increasing destination stride (the tile's
  // rows); B: the rest (batch).  I takes at least PERM_GROUP_MIN elements.
  // The destination's contiguous run (its unit-stride leg, then the legs
  // continuing it) is written either along I, in destination order, as far
  // as it lies inside I (I grown to take the unit-stride leg), or along O,
  // as far as it lies outside I (the run's legs kept out of I); the plan
  // with the longer run wins.  I grows further towards PERM_GROUP_I (at
  // most PERM_GROUP_IMAX) without breaking the chosen run.
  std::vector<int> by_d(r);
  for (int k = 0; k < r; ++k) by_d[k] = k;
  std::stable_sort(by_d.begin(), by_d.end(), [&](int a, int b) { return dstr[a] < dstr[b]; });
  const int fleg = by_d[0];
  std::vector<int> chain;  // the destination's contiguous run, fastest first
  if (dstr[fleg] == 1) {
    int64_t run = 1;
    for (;;) {
      int nxt = -1;
      for (int k = 0; k < r; ++k)
        if (dstr[k] == run && std::find(chain.begin(), chain.end(), k) == chain.end()) nxt = k;
      if (nxt < 0) break;
      chain.push_back(nxt);
      run *= dims[nxt];
    }
  }
  auto prod = [&](int from) {
    int64_t p = 1;
    for (int k = from; k < r; ++k) p *= dims[k];
    return p;
  };
  auto run_in = [&](int from) {  // run length along I = [from, r)
    int64_t p = 1;
    for (int k : chain) {
      if (k < from) break;
      p *= dims[k];
    }
    return p;
  };
  auto run_out = [&](int from) {  // run length along O (legs below from)
    int64_t p = 1;
    for (int k : chain) {
      if (k >= from) break;
      p *= dims[k];
    }
    return p;
  };
  int iI = r;
  while (iI > 0 && prod(iI) < PERM_GROUP_MIN) --iI;
  // plan along I: I reaches down to the unit-stride leg
  int iB = std::min(iI, fleg);
  const bool b_ok = prod(iB) <= PERM_GROUP_IMAX || iB == iI;
  if (b_ok)
    while (iB > 0 && prod(iB) < PERM_GROUP_I && prod(iB - 1) <= PERM_GROUP_IMAX) --iB;
  // plan along O: the run's legs stay out of I
  int iA = iI;
  if (fleg < iI) {
    std::vector<char> keep(r, 0);
    int64_t po = 1;
    for (int k : by_d) {
      if (po >= PERM_GROUP_O) break;
      if (k >= iA) continue;
      keep[k] = 1;
      po *= dims[k];
    }
    while (iA > 0 && prod(iA) < PERM_GROUP_I && prod(iA - 1) <= PERM_GROUP_IMAX && !keep[iA - 1]) --iA;
  }
  if (fleg >= iI || (b_ok && run_in(iB) > run_out(iA)))
    iI = iB;
  else
    iI = iA;
  const int64_t PI = prod(iI);
  // W: the part of the run inside I (the I legs are job legs 0..nI-1 in source order)
  int32_t wmask = 0;
  int64_t qw = 1;
  for (int k : chain) {
    if (k < iI) break;
    wmask |= 1 << (k - iI);
    qw *= dims[k];
  }
  // O group: remaining legs by increasing destination stride
  std::vector<int> rest;
  for (int k : by_d)
    if (k < iI) rest.push_back(k);
  std::vector<int> O, B;
  int64_t PO = 1;
  for (int k : rest) {
    if (PO < PERM_MAX_ROWS)
      O.push_back(k), PO *= dims[k];
    else
      B.push_back(k);
  }
  // order O legs so that the last one is the fastest in the destination
  std::sort(O.begin(), O.end(), [&](int a, int b) { return dstr[a] > dstr[b]; });
  PermJob j;
  std::memset(&j, 0, sizeof(j));
  j.src_off = src_off;
  j.dst_off = dst_off;
  j.sign = sign;
  int q = 0;
  for (int k = iI; k < r; ++k, ++q) {
    j.dim[q] = (int32_t)dims[k];
    j.sstr[q] = sstr[k];
    j.dstr[q] = dstr[k];
  }
  j.nI = r - iI;
  for (int k : O) {
    j.dim[q] = (int32_t)dims[k];
    j.sstr[q] = sstr[k];
    j.dstr[q] = dstr[k];
    ++q;
  }
  j.nO = (int32_t)O.size();
  int64_t PB = 1;
  for (int k : B) {
    j.dim[q] = (int32_t)dims[k];
    j.sstr[q] = sstr[k];
    j.dstr[q] = dstr[k];
    PB *= dims[k];
    ++q;
  }
  j.nB = (int32_t)B.size();
  j.PI = (int32_t)PI;
  j.PO = (int32_t)PO;
  j.PB = PB;

  // stores run along I when I holds the destination's unit-stride leg
  j.store_fast_i = fleg >= iI ? 1 : 0;
  j.wmask = wmask;
  j.qw = (int32_t)qw;
  j.iwrite = 0;
  {
    // the run's source strides equal its destination strides: q-th run
    // element = q-th source column of the run
    bool suf = wmask != 0;
    for (int q = 0; q < j.nI; ++q)
      if (wmask >> q & 1) suf = suf && j.sstr[q] == j.dstr[q];
    j.wsuf = suf ? 1 : 0;
  }
  jobs.push_back(j);
  (void)tiles;
}

int finalize_perm_jobs(std::vector<PermJob>& jobs, size_t es, int64_t* tiles, bool allow_staged) {
  const int64_t V = 16 / (int64_t)es;  // elements per 16 bytes
  bool staged = allow_staged && !jobs.empty();
  int64_t total = 0;
  for (const PermJob& j : jobs) total += (int64_t)j.PI * j.PO * j.PB;
  if (total < 65536) staged = false;  // tiny tensors: launch latency dominates, skip the staging ring
  for (PermJob& j : jobs) {
    bool ok = (j.PI % V == 0) && (j.src_off % V == 0);
    for (int q = j.nI; q < j.nI + j.nO + j.nB; ++q) ok = ok && (j.sstr[q] % V == 0);
    j.bulk_ok = ok ? 1 : 0;
    staged = staged && ok;
  }
  const int64_t te = PERM_TILE_BYTES / (int64_t)es;
  int64_t t = 0;
  for (PermJob& j : jobs) {
    j.vec4 = 0;
    // destination-order stores along I need the whole I group in one tile
    j.iwrite = staged && j.store_fast_i && j.wmask && j.PI <= te / 8 ? 1 : 0;
    if (staged) {
      // vector stores: the fastest destination leg along the store direction
      // has stride 1 and a dimension divisible by 4, every other destination
      // stride and the offset are multiples of 4 elements
      const int nl = j.nI + j.nO + j.nB;
      // (only along I: quads of O rows would read shared memory down a column)
      const int fast = j.nI - 1;
      bool v = j.store_fast_i && fast >= 0 && j.dst_off % 4 == 0 && j.dstr[fast] == 1 && j.dim[fast] % 4 == 0;
      for (int q = 0; q < nl; ++q)
        if (q != fast) v = v && j.dstr[q] % 4 == 0;
      j.vec4 = v ? 1 : 0;
    }
    if (j.iwrite) {
      // quads of the destination run: the run length and every other
      // destination stride are multiples of 4 elements
      const int nl = j.nI + j.nO + j.nB;
      bool v = j.dst_off % 4 == 0 && j.qw % 4 == 0;
      for (int q = 0; q < nl; ++q)
        if (!(q < j.nI && (j.wmask >> q & 1))) v = v && j.dstr[q] % 4 == 0;
      j.vec4 = v ? 1 : 0;
    }
    if (staged) {
      int64_t ti = j.iwrite ? j.PI : std::min<int64_t>(j.PI, te / 8);
      ti = (ti + V - 1) / V * V;
      int64_t tr = std::min<int64_t>(std::max<int64_t>(te / ti, 1), PERM_MAX_ROWS);
      tr = std::min<int64_t>(tr, j.PO);
      j.ti = (int32_t)ti;
      j.tr = (int32_t)tr;
    } else {
      j.ti = PERM_TI;
      j.tr = PERM_TO;
    }
    j.tiles_i = (int32_t)((j.PI + j.ti - 1) / j.ti);
    j.tiles_o = (int32_t)((j.PO + j.tr - 1) / j.tr);
    j.tile_begin = t;
    t += (int64_t)j.tiles_i * j.tiles_o * j.PB;
  }
  *tiles = t;
  return staged ? 1 : 0;
}

static cudaEvent_t take_event(ftn_ctx ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_begin(ftn_ctx ctx, const char* label, double bytes, double flops) {
  if (!ctx->prof_on) return -1;
  std::string full = ctx->prof_tag.empty() ? std::string(label) : ctx->prof_tag + "/" + label;
  ftn_prof_rec r{full, take_event(ctx), take_event(ctx), bytes, flops};
  cudaEventRecord(r.a, ctx->stream);
  ctx->prof.push_back(r);
  return (int)ctx->prof.size() - 1;
}

void prof_end(ftn_ctx ctx, int rec) {
  if (rec < 0 || rec >= (int)ctx->prof.size()) return;
  cudaEventRecord(ctx->prof[rec].b, ctx->stream);
}

static void prof_clear(ftn_ctx ctx) {
  for (auto& r : ctx->prof) {
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->prof.clear();
  ctx->prof_labels.clear();
}

}  // namespace ftn

using namespace ftn;

extern "C" {

const char* ftn_last_error(void) { return g_last_error.c_str(); }

ftn_status ftn_ctx_create(void* cuda_stream, ftn_alloc_fn alloc, ftn_free_fn free_fn, void* user, ftn_ctx* out) {
  if (!out) return set_error(FTN_EINVAL, "null out");
  if ((alloc == nullptr) != (free_fn == nullptr)) return set_error(FTN_EINVAL, "give both alloc and free or neither");
  int dev = 0;
  FTN_CUDA(cudaGetDevice(&dev));
  auto* c = new ftn_ctx_s();
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  c->device = dev;
  cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete c;
    return cuda_error(e, "cudaDeviceGetAttribute");
  }
  if (!alloc) {
    // library-owned buffers come from the device's stream-ordered pool; keep
    // freed memory pooled instead of returning it to the driver at every sync
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  c->dev_err = (int*)dev_alloc(c, 256);
  if (!c->dev_err) {
    delete c;
    return set_error(FTN_ENOMEM, "device allocation failed (error word)");
  }
  e = cudaMemsetAsync(c->dev_err, 0, 256, c->stream);
  if (e != cudaSuccess) {
    delete c;
    return cuda_error(e, "cudaMemsetAsync");
  }
  *out = c;
  return FTN_OK;
}

ftn_status ftn_ctx_destroy(ftn_ctx ctx) {
  if (!ctx) return FTN_OK;
  cudaStreamSynchronize(ctx->stream);
  prof_clear(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  ctx->ev_pool.clear();
  clear_plan_caches(ctx);
  dev_free(ctx, ctx->ws);
  dev_free(ctx, ctx->dev_err);
  release_cached_blocks(ctx);
  cudaStreamSynchronize(ctx->stream);
  for (void* p : ctx->graph_host) cudaFreeHost(p);
  delete ctx;
  return FTN_OK;
}

ftn_status ftn_ctx_set_stream(ftn_ctx ctx, void* cuda_stream) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  // cached blocks were freed in the old stream's order: let it finish first
  // (not while either stream is being captured: the cache is idle then, and
  // a synchronisation would break the capture)
  if ((cudaStream_t)cuda_stream != ctx->stream && !capturing((cudaStream_t)cuda_stream) && !capturing(ctx->stream))
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->stream = (cudaStream_t)cuda_stream;
  return FTN_OK;
}

ftn_status ftn_ctx_set_tuning(ftn_ctx ctx, int on) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  ctx->tune = on != 0;
  return FTN_OK;
}

ftn_status ftn_ctx_synchronize(ftn_ctx ctx) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  int err = 0;
  FTN_CUDA(cudaMemcpy(&err, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    FTN_CUDA(cudaMemset(ctx->dev_err, 0, sizeof(int)));
    return set_error(FTN_ETIMEOUT, "a device-side bounded wait timed out");
  }
  return FTN_OK;
}

ftn_status ftn_ctx_wait_selftest(ftn_ctx ctx, uint64_t limit_ns) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  if (limit_ns < 1000 || limit_ns > 10000000000ull)
    return set_error(FTN_EINVAL, "ftn_ctx_wait_selftest: limit_ns must lie in [1e3, 1e10]");
  return launch_wait_selftest(ctx, limit_ns);
}

int64_t ftn_ctx_launch_count(ftn_ctx ctx) { return ctx ? ctx->launches : 0; }

ftn_status ftn_ctx_profile(ftn_ctx ctx, int enable) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  if (enable) prof_clear(ctx);
  ctx->prof_on = enable != 0;
  return FTN_OK;
}

ftn_status ftn_ctx_profile_tag(ftn_ctx ctx, const char* tag) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  ctx->prof_tag = tag ? tag : "";
  return FTN_OK;
}

ftn_status ftn_ctx_profile_read(ftn_ctx ctx, int idx, const char** label, int64_t* launches, double* ms,
                                double* bytes, double* flops) {
  if (!ctx) return set_error(FTN_EINVAL, "null ctx");
  FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->prof_labels.clear();
  for (auto& r : ctx->prof)
    if (std::find(ctx->prof_labels.begin(), ctx->prof_labels.end(), r.label) == ctx->prof_labels.end())
      ctx->prof_labels.push_back(r.label);
  if (idx < 0 || idx >= (int)ctx->prof_labels.size()) return set_error(FTN_EINVAL, "no such profile label");
  const std::string& want = ctx->prof_labels[idx];
  int64_t n = 0;
  double t = 0, by = 0, fl = 0;
  for (auto& r : ctx->prof) {
    if (r.label != want) continue;
    float e = 0.f;
    FTN_CUDA(cudaEventElapsedTime(&e, r.a, r.b));
    ++n;
    t += e;
    by += r.bytes;
    fl += r.flops;
  }
  if (label) *label = ctx->prof_labels[idx].c_str();
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (bytes) *bytes = by;
  if (flops) *flops = fl;
  return FTN_OK;
}

ftn_status ftn_tensor_create(ftn_ctx ctx, int rank, const int32_t* d_even, const int32_t* d_odd, const uint8_t* dual,
                             int parity, ftn_dtype dtype, ftn_tensor* out) {
  return make_tensor(ctx, rank, d_even, d_odd, dual, parity, dtype, out);
}

ftn_status ftn_tensor_wrap(ftn_ctx ctx, int rank, const int32_t* d_even, const int32_t* d_odd, const uint8_t* dual,
                           int parity, ftn_dtype dtype, void* dev_data, ftn_tensor* out) {
  if (!ctx || !out) return set_error(FTN_EINVAL, "null argument");
  auto* t = new ftn_tensor_s();
  t->ctx = ctx;
  ftn_status st = fill_meta(t, rank, d_even, d_odd, dual, parity, dtype);
  if (st != FTN_OK) {
    delete t;
    return st;
  }
  if (!dev_data && t->numel > 0) {
    delete t;
    return set_error(FTN_EINVAL, "null device buffer");
  }
  if (((uintptr_t)dev_data) % dtype_size(dtype)) {
    delete t;
    return set_error(FTN_EINVAL, "device buffer not aligned to the element size");
  }
  t->data = dev_data;
  t->owned = false;
  *out = t;
  return FTN_OK;
}

ftn_status ftn_tensor_free(ftn_tensor t) {
  if (!t) return FTN_OK;
  if (t->owned) dev_free(t->ctx, t->data);
  delete t;
  return FTN_OK;
}

ftn_status ftn_tensor_info(ftn_tensor t, int* rank, int32_t* d_even, int32_t* d_odd, uint8_t* dual, int* parity,
                           ftn_dtype* dtype, int64_t* numel, void** dev_data) {
  if (!t) return set_error(FTN_EINVAL, "null tensor");
  if (rank) *rank = t->rank;
  for (int k = 0; k < t->rank; ++k) {
    if (d_even) d_even[k] = t->d0[k];
    if (d_odd) d_odd[k] = t->d1[k];
    if (dual) dual[k] = t->dual[k];
  }
  if (parity) *parity = t->parity;
  if (dtype) *dtype = t->dtype;
  if (numel) *numel = t->numel;
  if (dev_data) *dev_data = t->data;
  return FTN_OK;
}

ftn_status ftn_tensor_block_offsets(ftn_tensor t, int64_t* offsets, uint32_t* masks, int* nb) {
  if (!t) return set_error(FTN_EINVAL, "null tensor");
  int64_t n = nblocks(t->rank, t->parity);
  for (int64_t b = 0; b < n; ++b) {
    if (offsets) offsets[b] = t->offsets[b];
    if (masks) masks[b] = block_mask(t->rank, t->parity, b);
  }
  if (nb) *nb = (int)n;
  return FTN_OK;
}

ftn_status ftn_tensor_upload(ftn_ctx ctx, ftn_tensor t, const void* host) {
  if (!ctx || !t || (!host && t->numel)) return set_error(FTN_EINVAL, "null argument");
  if (t->numel)
    FTN_CUDA(cudaMemcpyAsync(t->data, host, (size_t)t->numel * dtype_size(t->dtype), cudaMemcpyHostToDevice,
                             ctx->stream));
  return FTN_OK;
}

ftn_status ftn_tensor_download(ftn_ctx ctx, ftn_tensor t, void* host) {
  if (!ctx || !t || (!host && t->numel)) return set_error(FTN_EINVAL, "null argument");
  if (t->numel)
    FTN_CUDA(cudaMemcpyAsync(host, t->data, (size_t)t->numel * dtype_size(t->dtype), cudaMemcpyDeviceToHost,
                             ctx->stream));
  return FTN_OK;
}

}  // extern "C"
