// Online verification service: many event streams, each an independent trace
// checked against the service's formula, with the submonitor tree kept on the
// GPU between chunks (the online mode of Algorithm 1, Sec. 4.2: repeated
// invocations update the tree and yield an evolving verdict).
//
// Continuous batching: rv_stream_push stages a chunk and returns at once; a
// worker thread repeatedly takes every staged chunk it can (at most one chunk
// per stream, so each chunk's verdict is the verdict of exactly its stream's
// prefix), copies them to the device in one batch and runs
//   k_s_ids       event -> dense ids of its binding and outer node, through
//                 device hash tables (new bindings spawn here, once: Sec. 3.3)
//   offline fold  the batch is grouped and folded by the offline kernels in
//                 streaming mode: each binding's map over the batch is applied
//                 to its stored state; verdict changes become count deltas of
//                 its outer node and of the stream's root
//   k_s_root      each chunk's stream root is valuated into a verdict record.
// Chunks that arrive while a batch runs wait for the next one.  Admission is
// by memory: a chunk is refused (RV_EAGAIN) when the staging budget or the
// worst-case binding capacity would be exceeded.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "profile.h"
#include "rv_device.cuh"

using namespace rvd;

void* rv_dev_alloc(size_t bytes);
void rv_dev_free(void* p);
rv_status rv_offline_stream_batch(const rv_formula* f, const uint64_t* key, const uint8_t* pred, uint64_t n,
                                  void* ws, size_t ws_bytes, const StreamState* ss, unsigned int* err_out,
                                  cudaStream_t s);
size_t rv_offline_stream_ws(const rv_formula* f, uint64_t n);

namespace {

constexpr uint32_t NO_ID = 0xFFFFFFFFu;
constexpr unsigned ERR_TABLE = 64;

struct Entry { unsigned long long k1; uint32_t k2; uint32_t id; };

struct ChunkDesc { uint64_t begin; uint32_t n; uint32_t stream; };

struct STables {
  Entry* bind;
  Entry* outer;
  uint64_t bind_mask, outer_mask;
  uint32_t bind_cap_ids, outer_cap_ids;
  unsigned int* counters;        // [0] next binding id, [1] next outer id
  StreamState ss;
};

__device__ __forceinline__ uint64_t hkey(uint64_t k1, uint32_t k2) {
  return mix64(k1 ^ ((uint64_t)k2 * 0x9E3779B97F4A7C15ull));
}

// id of (k1, k2), inserting it when absent; *fresh reports an insertion
__device__ uint32_t table_id(Entry* T, uint64_t mask, uint32_t cap_ids, unsigned int* counter, uint64_t k1,
                             uint32_t k2, bool* fresh, unsigned int* err) {
  uint64_t h = hkey(k1, k2) & mask;
  *fresh = false;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    volatile Entry* e = &T[h];
    unsigned long long cur = e->k1;
    if (cur == 0) {
      cur = atomicCAS((unsigned long long*)&T[h].k1, 0ull, (unsigned long long)k1);
      if (cur == 0) {
        const uint32_t id = atomicAdd(counter, 1u);
        e->k2 = k2;
        __threadfence();
        if (id >= cap_ids) { atomicOr(err, ERR_TABLE); e->id = NO_ID - 1; return NO_ID; }
        e->id = id;
        *fresh = true;
        return id;
      }
    }
    if (cur == k1) {
      uint32_t id;
      int spins = 0;
      while ((id = e->id) == NO_ID) {
        if (++spins > (1 << 24)) { atomicOr(err, (unsigned)ERR_SPIN); return NO_ID; }
      }
      __threadfence();
      if (id == NO_ID - 1) return NO_ID;
      if (e->k2 == k2) return id;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, ERR_TABLE);
  return NO_ID;
}

__global__ void k_s_init(Entry* T, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    T[i].k1 = 0;
    T[i].k2 = 0;
    T[i].id = NO_ID;
  }
}

// event -> (outer id << 32) | binding id  (two quantifiers)  or  binding id (one)
__global__ void k_s_ids(STables tb, const ChunkDesc* chunks, int nchunks, const void* keys, int key_bits, int nq,
                        const uint8_t* pred, int n_letters, uint64_t n, uint64_t* ids, unsigned int* err) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nchunks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunks[mid].begin <= i) lo = mid; else hi = mid - 1;
  }
  const uint32_t s = chunks[lo].stream;
  if (pred[i] >= n_letters) atomicOr(err, (unsigned)ERR_LETTER);
  const uint64_t key = key_bits == 64 ? ((const uint64_t*)keys)[i] : ((const uint32_t*)keys)[i];
  bool fresh;
  if (nq == 2) {
    const uint64_t k1 = (((uint64_t)s << 32) | (key >> 32)) + 1;
    const uint32_t o = table_id(tb.outer, tb.outer_mask, tb.outer_cap_ids, &tb.counters[1], k1, 0, &fresh, err);
    if (o != NO_ID && fresh) {
      tb.ss.ostream[o] = (uint16_t)s;
      tb.ss.overdict[o] = 0xFF;
      for (int v = 0; v < 6; ++v) tb.ss.ocounts[(uint64_t)o * 6 + v] = 0;
    }
    const uint32_t b = table_id(tb.bind, tb.bind_mask, tb.bind_cap_ids, &tb.counters[0], k1,
                                (uint32_t)(key & 0xFFFFFFFFull), &fresh, err);
    if (b != NO_ID && fresh) tb.ss.bstate[b] = 0;
    ids[i] = ((uint64_t)(o == NO_ID ? 0 : o) << 32) | (b == NO_ID ? 0 : b);
  } else {
    const uint64_t k1 = (((uint64_t)s << 32) | (key & 0xFFFFFFFFull)) + 1;
    const uint32_t b = table_id(tb.bind, tb.bind_mask, tb.bind_cap_ids, &tb.counters[0], k1, 0, &fresh, err);
    if (b != NO_ID && fresh) { tb.ss.bstate[b] = 0; tb.ss.bstream[b] = (uint16_t)s; }
    ids[i] = b == NO_ID ? 0 : b;
  }
}

struct SRecord { uint32_t stream; int32_t root; uint64_t counts[6]; };

__global__ void k_s_root(const ChunkDesc* chunks, int nchunks, rv_quant q, const unsigned long long* root,
                         SRecord* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  const uint32_t s = chunks[c].stream;
  uint64_t v[6];
  for (int k = 0; k < 6; ++k) v[k] = root[s * 6 + k];
  SRecord r;
  r.stream = s;
  r.root = rvv::valuate(q.kind, q.op, q.num, q.den, v);
  for (int k = 0; k < 6; ++k) r.counts[k] = v[k];
  out[c] = r;
}

#define SCU(call)                                                                               \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return rv_fail(RV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

typedef std::chrono::steady_clock Clock;

struct Staged {
  rv_stream* st;
  uint32_t stream;
  uint64_t ticket;
  std::vector<unsigned char> key;
  std::vector<uint8_t> pred;
  uint64_t n;
  uint64_t events_after;      // the stream's events up to and including this chunk
  Clock::time_point t_push;
};

}  // namespace

struct rv_stream {
  rv_service* svc;
  uint32_t id;
  uint64_t next_ticket = 1;
  uint64_t events = 0;            // events admitted so far
  bool closed = false;
  bool in_flight = false;
  std::deque<rv_stream_verdict> out;
};

struct rv_service {
  rv_formula f;
  rv_service_cfg cfg;
  int key_bytes;
  // device
  void* dmem = nullptr;
  STables tb{};
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  unsigned char* d_keys = nullptr;
  uint8_t* d_pred = nullptr;
  uint64_t* d_ids = nullptr;
  ChunkDesc* d_chunks = nullptr;
  SRecord* d_rec = nullptr;
  unsigned int* d_err = nullptr;
  // host pinned
  unsigned char* h_keys = nullptr;
  uint8_t* h_pred = nullptr;
  ChunkDesc* h_chunks = nullptr;
  SRecord* h_rec = nullptr;
  unsigned int* h_err = nullptr;
  unsigned int* h_counters = nullptr;
  cudaStream_t cs = nullptr;
  int device = 0;
  // host state
  std::mutex mu;
  std::condition_variable cv_work, cv_out;
  std::deque<Staged> pending;
  std::vector<rv_stream*> streams;
  uint64_t staged_events = 0;
  uint64_t reserved_bindings = 0;   // worst-case bindings of admitted chunks
  uint64_t bindings_used = 0, outer_used = 0;
  uint64_t batches = 0, admitted = 0, refused = 0, processed_events = 0;
  bool stop = false;
  rv_status worker_status = RV_OK;
  std::thread worker;
};

namespace {

void publish(rv_service* S, std::vector<Staged>& batch, rv_status st, Clock::time_point t_done) {
  std::lock_guard<std::mutex> lk(S->mu);
  for (size_t c = 0; c < batch.size(); ++c) {
    Staged& ch = batch[c];
    ch.st->in_flight = false;
    S->staged_events -= ch.n;
    if (ch.st->closed) continue;
    rv_stream_verdict v;
    memset(&v, 0, sizeof v);
    v.ticket = ch.ticket;
    v.status = st;
    if (st == RV_OK) {
      v.root = S->h_rec[c].root;
      for (int k = 0; k < 6; ++k) v.root_counts[k] = S->h_rec[c].counts[k];
    }
    v.events = ch.events_after;
    v.latency_us = std::chrono::duration<double, std::micro>(t_done - ch.t_push).count();
    ch.st->out.push_back(v);
  }
  S->cv_out.notify_all();
  S->cv_work.notify_all();
}

rv_status run_batch(rv_service* S, std::vector<Staged>& batch) {
  uint64_t n = 0;
  for (size_t c = 0; c < batch.size(); ++c) {
    S->h_chunks[c] = ChunkDesc{n, (uint32_t)batch[c].n, batch[c].stream};
    memcpy(S->h_keys + n * S->key_bytes, batch[c].key.data(), batch[c].n * S->key_bytes);
    memcpy(S->h_pred + n, batch[c].pred.data(), batch[c].n);
    n += batch[c].n;
  }
  const int nc = (int)batch.size();
  SCU(cudaMemcpyAsync(S->d_chunks, S->h_chunks, nc * sizeof(ChunkDesc), cudaMemcpyHostToDevice, S->cs));
  SCU(cudaMemcpyAsync(S->d_keys, S->h_keys, n * S->key_bytes, cudaMemcpyHostToDevice, S->cs));
  SCU(cudaMemcpyAsync(S->d_pred, S->h_pred, n, cudaMemcpyHostToDevice, S->cs));
  SCU(cudaMemsetAsync(S->d_err, 0, 4, S->cs));
  if (n) {
    RV_LAUNCH("k_s_ids", k_s_ids, (unsigned)((n + 255) / 256), 256, 0, S->cs, S->tb, S->d_chunks, nc, S->d_keys,
              S->f.key_bits, S->f.n_quant, S->d_pred, S->f.n_letters, n, S->d_ids, S->d_err);
    rv_status st = rv_offline_stream_batch(&S->f, S->d_ids, S->d_pred, n, S->ws, S->ws_bytes, &S->tb.ss,
                                           S->d_err + 1, S->cs);
    if (st) return st;
  }
  RV_LAUNCH("k_s_root", k_s_root, (nc + 63) / 64, 64, 0, S->cs, S->d_chunks, nc, S->f.q[0], S->tb.ss.root, S->d_rec);
  SCU(cudaMemcpyAsync(S->h_rec, S->d_rec, nc * sizeof(SRecord), cudaMemcpyDeviceToHost, S->cs));
  SCU(cudaMemcpyAsync(S->h_err, S->d_err, 8, cudaMemcpyDeviceToHost, S->cs));
  SCU(cudaMemcpyAsync(S->h_counters, S->tb.counters, 8, cudaMemcpyDeviceToHost, S->cs));
  SCU(cudaStreamSynchronize(S->cs));
  const unsigned e = S->h_err[0] | S->h_err[1];
  if (e & ERR_LETTER) return rv_fail(RV_EINVAL, "predicate code out of range in a streamed chunk");
  if (e & ERR_TABLE) return rv_fail(RV_ENOMEM, "binding table full");
  if (e) return rv_fail(RV_EINTERNAL, "device status 0x%x", e);
  return RV_OK;
}

void worker_main(rv_service* S) {
  cudaSetDevice(S->device);
  std::vector<Staged> batch;
  while (true) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->stop && S->pending.empty()) return;
      uint64_t total = 0;
      std::vector<char> taken(S->streams.size() + 1, 0);
      for (auto it = S->pending.begin(); it != S->pending.end();) {
        const uint32_t sid = it->stream;
        if (it->st->closed) {                       // dropped with its stream
          S->staged_events -= it->n;
          S->reserved_bindings -= it->n;
          it = S->pending.erase(it);
          continue;
        }
        if (taken[sid] || it->st->in_flight || total + it->n > S->cfg.max_batch_events) { ++it; continue; }
        taken[sid] = 1;
        it->st->in_flight = true;
        total += it->n;
        batch.push_back(std::move(*it));
        it = S->pending.erase(it);
      }
    }
    if (batch.empty()) continue;
    rv_status st = run_batch(S, batch);
    const Clock::time_point t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      uint64_t n = 0;
      for (auto& c : batch) n += c.n;
      S->reserved_bindings -= n;
      S->bindings_used = S->h_counters[0];
      S->outer_used = S->h_counters[1];
      S->batches += 1;
      S->processed_events += n;
      if (st) S->worker_status = st;
    }
    publish(S, batch, st, t_done);
  }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

extern "C" rv_status rv_service_open(const rv_formula* f, const rv_service_cfg* cfg, rv_service** out) {
  if (!f || !out) return rv_fail(RV_EINVAL, "null argument");
  *out = nullptr;
  if (f->n_quant < 1 || f->n_quant > 2) return rv_fail(RV_EUNSUPPORTED, "streaming needs one or two quantifiers");
  if (f->n_quant == 1 && f->key_bits != 32) return rv_fail(RV_EUNSUPPORTED, "one-quantifier streams use 32-bit keys");
  rv_service* S = new (std::nothrow) rv_service();
  if (!S) return rv_fail(RV_ENOMEM, "out of host memory");
  S->f = *f;
  rv_service_cfg c = cfg ? *cfg : rv_service_cfg{};
  if (!c.max_bindings) c.max_bindings = 1 << 24;
  if (!c.max_outer) c.max_outer = f->n_quant == 2 ? (1 << 22) : 1;
  if (!c.max_batch_events) c.max_batch_events = 1 << 22;
  if (!c.max_staged_events) c.max_staged_events = 1 << 25;
  if (!c.max_streams) c.max_streams = 64;
  if (c.max_streams > 65535 || c.max_bindings > 0xFFFFFF00ull || c.max_outer > 0xFFFFFF00ull)
    return delete S, rv_fail(RV_EINVAL, "service limits out of range");
  S->cfg = c;
  S->key_bytes = f->key_bits / 8;
  cudaGetDevice(&S->device);
  const uint64_t bcap = pow2_at_least(c.max_bindings * 2), ocap = pow2_at_least(c.max_outer * 2);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = a256(off + bytes); return r; };
  const size_t o_bind = take(bcap * sizeof(Entry)), o_outer = take(ocap * sizeof(Entry));
  const size_t o_bstate = take(c.max_bindings), o_bverd = take(c.max_bindings), o_bstream = take(c.max_bindings * 2);
  const size_t o_ocnt = take(c.max_outer * 24), o_overd = take(c.max_outer), o_ostream = take(c.max_outer * 2);
  const size_t o_root = take((size_t)c.max_streams * 6 * 8), o_ctr = take(16);
  const size_t o_keys = take(c.max_batch_events * S->key_bytes), o_pred = take(c.max_batch_events);
  const size_t o_ids = take(c.max_batch_events * 8), o_chunks = take((size_t)c.max_streams * sizeof(ChunkDesc));
  const size_t o_rec = take((size_t)c.max_streams * sizeof(SRecord)), o_err = take(16);
  S->ws_bytes = rv_offline_stream_ws(f, c.max_batch_events);
  const size_t o_ws = take(S->ws_bytes);
  S->dmem = rv_dev_alloc(off);
  if (!S->dmem) { delete S; return rv_fail(RV_ENOMEM, "cannot allocate %zu bytes of service memory", off); }
  unsigned char* D = (unsigned char*)S->dmem;
  S->tb.bind = (Entry*)(D + o_bind);
  S->tb.outer = (Entry*)(D + o_outer);
  S->tb.bind_mask = bcap - 1;
  S->tb.outer_mask = ocap - 1;
  S->tb.bind_cap_ids = (uint32_t)c.max_bindings;
  S->tb.outer_cap_ids = (uint32_t)c.max_outer;
  S->tb.counters = (unsigned int*)(D + o_ctr);
  S->tb.ss.bstate = D + o_bstate;
  S->tb.ss.bverdict = D + o_bverd;
  S->tb.ss.bstream = (uint16_t*)(D + o_bstream);
  S->tb.ss.ocounts = (uint32_t*)(D + o_ocnt);
  S->tb.ss.overdict = D + o_overd;
  S->tb.ss.ostream = (uint16_t*)(D + o_ostream);
  S->tb.ss.root = (unsigned long long*)(D + o_root);
  S->d_keys = D + o_keys;
  S->d_pred = D + o_pred;
  S->d_ids = (uint64_t*)(D + o_ids);
  S->d_chunks = (ChunkDesc*)(D + o_chunks);
  S->d_rec = (SRecord*)(D + o_rec);
  S->d_err = (unsigned int*)(D + o_err);
  S->ws = D + o_ws;
  auto fail = [&](rv_status s2) { rv_service_close(S); return s2; };
  if (cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking) != cudaSuccess) return fail(rv_fail(RV_ECUDA, "stream"));
  if (cudaMallocHost(&S->h_keys, c.max_batch_events * S->key_bytes) != cudaSuccess ||
      cudaMallocHost(&S->h_pred, c.max_batch_events) != cudaSuccess ||
      cudaMallocHost(&S->h_chunks, (size_t)c.max_streams * sizeof(ChunkDesc)) != cudaSuccess ||
      cudaMallocHost(&S->h_rec, (size_t)c.max_streams * sizeof(SRecord)) != cudaSuccess ||
      cudaMallocHost(&S->h_err, 16) != cudaSuccess || cudaMallocHost(&S->h_counters, 16) != cudaSuccess)
    return fail(rv_fail(RV_ENOMEM, "cannot allocate pinned staging"));
  k_s_init<<<1024, 256, 0, S->cs>>>(S->tb.bind, bcap);
  k_s_init<<<1024, 256, 0, S->cs>>>(S->tb.outer, ocap);
  if (cudaMemsetAsync(S->tb.counters, 0, 16, S->cs) != cudaSuccess ||
      cudaMemsetAsync(S->tb.ss.root, 0, (size_t)c.max_streams * 48, S->cs) != cudaSuccess ||
      cudaStreamSynchronize(S->cs) != cudaSuccess)
    return fail(rv_fail(RV_ECUDA, "service initialisation failed"));
  S->worker = std::thread(worker_main, S);
  *out = S;
  return RV_OK;
}

extern "C" rv_status rv_service_close(rv_service* S) {
  if (!S) return RV_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (rv_stream* st : S->streams) delete st;
  if (S->cs) { cudaStreamSynchronize(S->cs); cudaStreamDestroy(S->cs); }
  if (S->h_keys) cudaFreeHost(S->h_keys);
  if (S->h_pred) cudaFreeHost(S->h_pred);
  if (S->h_chunks) cudaFreeHost(S->h_chunks);
  if (S->h_rec) cudaFreeHost(S->h_rec);
  if (S->h_err) cudaFreeHost(S->h_err);
  if (S->h_counters) cudaFreeHost(S->h_counters);
  if (S->dmem) rv_dev_free(S->dmem);
  delete S;
  return RV_OK;
}

extern "C" rv_status rv_stream_open(rv_service* S, rv_stream** out) {
  if (!S || !out) return rv_fail(RV_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if ((int)S->streams.size() >= S->cfg.max_streams) return rv_fail(RV_EAGAIN, "all %d stream slots are in use", S->cfg.max_streams);
  rv_stream* st = new (std::nothrow) rv_stream();
  if (!st) return rv_fail(RV_ENOMEM, "out of host memory");
  st->svc = S;
  st->id = (uint32_t)S->streams.size();
  S->streams.push_back(st);
  *out = st;
  return RV_OK;
}

extern "C" rv_status rv_stream_push(rv_stream* st, const rv_trace* chunk, uint64_t* ticket) {
  if (!st || !chunk || (chunk->n && (!chunk->key || !chunk->pred))) return rv_fail(RV_EINVAL, "null argument");
  rv_service* S = st->svc;
  if (chunk->n > S->cfg.max_batch_events) return rv_fail(RV_EINVAL, "chunk larger than max_batch_events");
  if (chunk->ts)
    for (uint64_t i = 1; i < chunk->n; ++i)
      if (chunk->ts[i] < chunk->ts[i - 1]) return rv_fail(RV_EINVAL, "timestamps decrease inside the chunk");
  for (uint64_t i = 0; i < chunk->n; ++i)
    if (chunk->pred[i] >= S->f.n_letters) return rv_fail(RV_EINVAL, "predicate code %u out of range at %llu",
                                                         (unsigned)chunk->pred[i], (unsigned long long)i);
  Staged sc;
  sc.st = st;
  sc.stream = st->id;
  sc.n = chunk->n;
  sc.t_push = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (st->closed) return rv_fail(RV_EINVAL, "stream is closed");
    if (S->worker_status != RV_OK) return rv_fail(S->worker_status, "service failed earlier: %s", rv_last_error());
    // admission by memory: staging budget and worst-case new bindings
    const uint64_t inner_cap = S->cfg.max_bindings, outer_cap = S->cfg.max_outer;
    if (S->staged_events + chunk->n > S->cfg.max_staged_events ||
        S->bindings_used + S->reserved_bindings + chunk->n > inner_cap ||
        (S->f.n_quant == 2 && S->outer_used + S->reserved_bindings + chunk->n > outer_cap)) {
      S->refused += 1;
      return rv_fail(RV_EAGAIN, "chunk not admitted: memory budget");
    }
    S->staged_events += chunk->n;
    S->reserved_bindings += chunk->n;
    sc.ticket = st->next_ticket++;
    st->events += chunk->n;
    sc.events_after = st->events;
    S->admitted += 1;
  }
  sc.key.assign((const unsigned char*)chunk->key, (const unsigned char*)chunk->key + chunk->n * S->key_bytes);
  sc.pred.assign(chunk->pred, chunk->pred + chunk->n);
  const uint64_t tk = sc.ticket;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->pending.push_back(std::move(sc));
  }
  S->cv_work.notify_one();
  if (ticket) *ticket = tk;
  return RV_OK;
}

extern "C" rv_status rv_stream_poll(rv_stream* st, rv_stream_verdict* out, int max, int* n, int timeout_us) {
  if (!st || !n || (max > 0 && !out)) return rv_fail(RV_EINVAL, "null argument");
  rv_service* S = st->svc;
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&] { return !st->out.empty() || S->worker_status != RV_OK; };
  if (!ready() && timeout_us > 0)
    S->cv_out.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
  int k = 0;
  while (k < max && !st->out.empty()) { out[k++] = st->out.front(); st->out.pop_front(); }
  *n = k;
  if (k == 0) {
    if (S->worker_status != RV_OK) return rv_fail(S->worker_status, "service failed: %s", rv_last_error());
    return rv_fail(RV_ETIMEOUT, "no verdict within %d us", timeout_us);
  }
  return RV_OK;
}

extern "C" rv_status rv_stream_close(rv_stream* st) {
  if (!st) return RV_OK;
  rv_service* S = st->svc;
  std::lock_guard<std::mutex> lk(S->mu);
  st->closed = true;    // queued chunks are dropped; a chunk in flight completes unseen
  st->out.clear();
  return RV_OK;
}

extern "C" rv_status rv_service_stats(rv_service* S, rv_service_counters* out) {
  if (!S || !out) return rv_fail(RV_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out->batches = S->batches;
  out->admitted = S->admitted;
  out->refused = S->refused;
  out->events = S->processed_events;
  out->bindings = S->bindings_used;
  out->outer_nodes = S->outer_used;
  out->staged_events = S->staged_events;
  return RV_OK;
}
