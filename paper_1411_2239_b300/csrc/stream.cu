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
#include <atomic>
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
constexpr unsigned long long TOMB = ~0ull;   // a retired entry: probes go on past it, inserts may reuse it
constexpr int CLAIM_TRIES = 64;

struct Entry { unsigned long long k1; uint32_t k2; uint32_t id; };

struct ChunkDesc { uint64_t begin; uint32_t n; uint32_t stream; };

// counters[0]: next fresh binding id, [1]: next fresh outer id,
// counters[2], [3]: ids on the binding / outer free lists (signed)
struct STables {
  Entry* bind;
  Entry* outer;
  uint64_t bind_mask, outer_mask;
  uint32_t bind_cap_ids, outer_cap_ids;
  unsigned int* counters;
  uint32_t* free_bind;           // ids of retired bindings
  uint32_t* free_outer;          // ids of retired outer nodes
  StreamState ss;
};

__device__ __forceinline__ uint64_t hkey(uint64_t k1, uint32_t k2) {
  return mix64(k1 ^ ((uint64_t)k2 * 0x9E3779B97F4A7C15ull));
}

// wait (bounded) until the entry's id is published; NO_ID on a failed insert
__device__ __forceinline__ uint32_t entry_id(volatile Entry* e, unsigned int* err) {
  uint32_t id;
  int spins = 0;
  while ((id = e->id) == NO_ID) {
    if (++spins > (1 << 24)) { atomicOr(err, (unsigned)ERR_SPIN); return NO_ID - 1; }
  }
  __threadfence();
  return id;
}

// a new entry's id: a retired one from the free list, else a fresh one
__device__ __forceinline__ uint32_t new_id(unsigned int* counter, int* free_n, const uint32_t* free_ids) {
  const int t = atomicSub(free_n, 1);
  if (t > 0) return free_ids[t - 1];
  atomicAdd(free_n, 1);
  return atomicAdd(counter, 1u);
}

// id of (k1, k2), inserting it when absent; *fresh reports an insertion.
// Entries are only added while a batch runs (retired ones become TOMB between
// batches), so a key is searched over its whole probe chain first; only when
// it is absent does the inserter claim the chain's first free entry (a
// tombstone, else the empty entry that ended the search) with a CAS from that
// entry's free value.  Every inserter of one key targets the same first free
// entry, so exactly one claims it; a loser that finds another key there
// searches again.
__device__ uint32_t table_id(Entry* T, uint64_t mask, uint32_t cap_ids, unsigned int* counter, int* free_n,
                             const uint32_t* free_ids, uint64_t k1, uint32_t k2, bool* fresh, unsigned int* err) {
  *fresh = false;
  const uint64_t h0 = hkey(k1, k2) & mask;
  for (int attempt = 0; attempt < CLAIM_TRIES; ++attempt) {
    uint64_t h = h0, target = ~0ull;
    unsigned long long expect = 0;
    for (uint64_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
      volatile Entry* e = &T[h];
      const unsigned long long cur = e->k1;
      if (cur == TOMB) {
        if (target == ~0ull) { target = h; expect = TOMB; }
        continue;
      }
      if (cur == 0) {
        if (target == ~0ull) { target = h; expect = 0; }
        break;
      }
      if (cur == k1) {
        const uint32_t id = entry_id(e, err);
        if (id == NO_ID - 1) return NO_ID;
        if (e->k2 == k2) return id;
      }
    }
    if (target == ~0ull) break;                       // no free entry at all
    const unsigned long long prev = atomicCAS(&T[target].k1, expect, (unsigned long long)k1);
    if (prev == expect) {
      volatile Entry* e = &T[target];
      const uint32_t id = new_id(counter, free_n, free_ids);
      e->k2 = k2;
      __threadfence();
      if (id >= cap_ids) { atomicOr(err, ERR_TABLE); e->id = NO_ID - 1; return NO_ID; }
      e->id = id;
      *fresh = true;
      return id;
    }
    if (prev == k1) {                                  // another inserter with our k1 got there first
      volatile Entry* e = &T[target];
      const uint32_t id = entry_id(e, err);
      if (id == NO_ID - 1) return NO_ID;
      if (e->k2 == k2) return id;
    }
  }
  atomicOr(err, ERR_TABLE);
  return NO_ID;
}

// between batches: every entry of stream s becomes a tombstone and its id goes
// to the free list; the stream's root counts restart from zero
__global__ void k_s_retire(Entry* T, uint64_t n, uint32_t s, uint32_t cap_ids, int* free_n, uint32_t* free_ids,
                           unsigned long long* root) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long k1 = T[i].k1;
    if (k1 == 0 || k1 == TOMB || ((k1 - 1) >> 32) != s) continue;
    const uint32_t id = T[i].id;
    if (id < cap_ids) free_ids[atomicAdd(free_n, 1)] = id;
    T[i].id = NO_ID;
    T[i].k2 = 0;
    T[i].k1 = TOMB;
  }
  if (root && blockIdx.x == 0 && threadIdx.x < 6) root[(uint64_t)s * 6 + threadIdx.x] = 0;
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
    const uint32_t o = table_id(tb.outer, tb.outer_mask, tb.outer_cap_ids, &tb.counters[1], (int*)&tb.counters[3],
                                tb.free_outer, k1, 0, &fresh, err);
    if (o != NO_ID && fresh) {
      tb.ss.ostream[o] = (uint16_t)s;
      tb.ss.overdict[o] = 0xFF;
      for (int v = 0; v < 6; ++v) tb.ss.ocounts[(uint64_t)o * 6 + v] = 0;
    }
    const uint32_t b = table_id(tb.bind, tb.bind_mask, tb.bind_cap_ids, &tb.counters[0], (int*)&tb.counters[2],
                                tb.free_bind, k1, (uint32_t)(key & 0xFFFFFFFFull), &fresh, err);
    if (b != NO_ID && fresh) tb.ss.bstate[b] = 0;
    ids[i] = ((uint64_t)(o == NO_ID ? 0 : o) << 32) | (b == NO_ID ? 0 : b);
  } else {
    const uint64_t k1 = (((uint64_t)s << 32) | (key & 0xFFFFFFFFull)) + 1;
    const uint32_t b = table_id(tb.bind, tb.bind_mask, tb.bind_cap_ids, &tb.counters[0], (int*)&tb.counters[2],
                                tb.free_bind, k1, 0, &fresh, err);
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

// one of the two staging buffers: batch k uses buffer k % 2, so the host copy
// and the host->device copy of the next batch overlap this batch's kernels
struct Buf {
  unsigned char* h_keys = nullptr;   // pinned
  uint8_t* h_pred = nullptr;
  ChunkDesc* h_chunks = nullptr;
  SRecord* h_rec = nullptr;
  unsigned int* h_err = nullptr;     // [0] id kernel, [1] fold
  unsigned int* h_counters = nullptr;
  unsigned char* d_keys = nullptr;   // device
  uint8_t* d_pred = nullptr;
  ChunkDesc* d_chunks = nullptr;
  cudaEvent_t copied = nullptr, done = nullptr;
};

struct InFlight {
  std::vector<Staged> batch;
  int buf = 0;
  rv_status launch = RV_OK;
};

}  // namespace

struct rv_stream {
  rv_service* svc;
  uint32_t id;
  uint64_t next_ticket = 1;
  uint64_t events = 0;            // events admitted so far
  bool closed = false;
  bool failed = false;            // a batch carrying one of its chunks failed on the device
  int in_flight = 0;              // its chunks inside launched, unpublished batches
  std::deque<rv_stream_verdict> out;
};

struct rv_service {
  rv_formula f;
  rv_service_cfg cfg;
  int key_bytes;
  // device
  void* dmem = nullptr;
  STables tb{};
  uint64_t bcap = 0, ocap = 0;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  uint64_t* d_ids = nullptr;
  SRecord* d_rec = nullptr;
  unsigned int* d_err = nullptr;
  Buf buf[2];
  unsigned int* h_retire_counters = nullptr;   // pinned
  cudaStream_t cs = nullptr;         // kernels, in batch order
  cudaStream_t cp = nullptr;         // host->device copies of the next batch
  int device = 0;
  // host state
  std::mutex mu;
  std::condition_variable cv_work, cv_out;
  std::deque<Staged> pending;
  std::vector<rv_stream*> slots;     // by stream id; nullptr: free
  std::vector<uint32_t> free_slots;
  std::vector<rv_stream*> to_retire; // closed streams whose state is still on the device
  uint64_t staged_events = 0;
  uint64_t reserved_bindings = 0;    // worst-case bindings of admitted chunks
  uint64_t bindings_used = 0, outer_used = 0;
  uint64_t batches = 0, admitted = 0, refused = 0, processed_events = 0, retired = 0;
  bool stop = false;
  rv_status fatal = RV_OK;           // CUDA failures only: the context may be unusable
  std::thread worker;
};

namespace {

#define SCU_F(call)                                                                              \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return rv_fail(RV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

void publish(rv_service* S, InFlight& b, rv_status st, Clock::time_point t_done) {
  std::lock_guard<std::mutex> lk(S->mu);
  const Buf& B = S->buf[b.buf];
  uint64_t n = 0;
  for (size_t c = 0; c < b.batch.size(); ++c) {
    Staged& ch = b.batch[c];
    n += ch.n;
    ch.st->in_flight -= 1;
    S->staged_events -= ch.n;
    if (st != RV_OK) ch.st->failed = true;      // its device state is no longer trustworthy
    if (ch.st->closed) continue;
    rv_stream_verdict v;
    memset(&v, 0, sizeof v);
    v.ticket = ch.ticket;
    v.status = st;
    if (st == RV_OK) {
      v.root = B.h_rec[c].root;
      for (int k = 0; k < 6; ++k) v.root_counts[k] = B.h_rec[c].counts[k];
    }
    v.events = ch.events_after;
    v.latency_us = std::chrono::duration<double, std::micro>(t_done - ch.t_push).count();
    ch.st->out.push_back(v);
  }
  S->reserved_bindings -= n;
  if (st == RV_OK || st != RV_ECUDA) {
    const int free_b = (int)B.h_counters[2], free_o = (int)B.h_counters[3];
    S->bindings_used = B.h_counters[0] - (uint64_t)std::max(0, free_b);
    S->outer_used = B.h_counters[1] - (uint64_t)std::max(0, free_o);
  }
  S->batches += 1;
  S->processed_events += n;
  if (st == RV_ECUDA) S->fatal = st;
  S->cv_out.notify_all();
  S->cv_work.notify_all();
}

// stage batch b into its buffer and queue its copies and kernels
// Copies of a batch's chunks into the pinned staging buffer.  A large batch
// is copied by several host threads, each taking pieces of at most PIECE
// bytes in turn: one thread copies about 10 GB/s, and a batch of a few
// million events would otherwise hold its verdicts back by milliseconds.
struct CopyItem { unsigned char* dst; const unsigned char* src; size_t bytes; };
constexpr size_t PIECE = 1u << 20;
constexpr size_t PARALLEL_FROM = 4u << 20;   // smaller batches: one thread
constexpr unsigned COPY_THREADS = 4;

void copy_pieces(const std::vector<CopyItem>& items, size_t total) {
  if (total < PARALLEL_FROM) {
    for (const CopyItem& it : items) memcpy(it.dst, it.src, it.bytes);
    return;
  }
  std::vector<CopyItem> pieces;
  for (const CopyItem& it : items)
    for (size_t o = 0; o < it.bytes; o += PIECE) pieces.push_back({it.dst + o, it.src + o, std::min(PIECE, it.bytes - o)});
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t k = next++; k < pieces.size(); k = next++) memcpy(pieces[k].dst, pieces[k].src, pieces[k].bytes);
  };
  std::vector<std::thread> helpers;
  for (unsigned t = 1; t < COPY_THREADS; ++t) helpers.emplace_back(work);
  work();
  for (std::thread& h : helpers) h.join();
}

rv_status launch_batch(rv_service* S, InFlight& b) {
  Buf& B = S->buf[b.buf];
  uint64_t n = 0;
  std::vector<CopyItem> items;
  size_t total = 0;
  for (size_t c = 0; c < b.batch.size(); ++c) {
    Staged& ch = b.batch[c];
    B.h_chunks[c] = ChunkDesc{n, (uint32_t)ch.n, ch.stream};
    items.push_back({B.h_keys + n * S->key_bytes, ch.key.data(), ch.n * S->key_bytes});
    items.push_back({B.h_pred + n, ch.pred.data(), ch.n});
    total += ch.n * (S->key_bytes + 1);
    n += ch.n;
  }
  copy_pieces(items, total);
  const int nc = (int)b.batch.size();
  SCU_F(cudaMemcpyAsync(B.d_chunks, B.h_chunks, nc * sizeof(ChunkDesc), cudaMemcpyHostToDevice, S->cp));
  if (n) {
    SCU_F(cudaMemcpyAsync(B.d_keys, B.h_keys, n * S->key_bytes, cudaMemcpyHostToDevice, S->cp));
    SCU_F(cudaMemcpyAsync(B.d_pred, B.h_pred, n, cudaMemcpyHostToDevice, S->cp));
  }
  SCU_F(cudaEventRecord(B.copied, S->cp));
  SCU_F(cudaStreamWaitEvent(S->cs, B.copied, 0));
  SCU_F(cudaMemsetAsync(S->d_err, 0, 8, S->cs));
  if (n) {
    RV_LAUNCH("k_s_ids", k_s_ids, (unsigned)((n + 255) / 256), 256, 0, S->cs, S->tb, B.d_chunks, nc, B.d_keys,
              S->f.key_bits, S->f.n_quant, B.d_pred, S->f.n_letters, n, S->d_ids, S->d_err);
    rv_status st = rv_offline_stream_batch(&S->f, S->d_ids, B.d_pred, n, S->ws, S->ws_bytes, &S->tb.ss,
                                           S->d_err + 1, S->cs);
    if (st) return st;
  }
  RV_LAUNCH("k_s_root", k_s_root, (nc + 63) / 64, 64, 0, S->cs, B.d_chunks, nc, S->f.q[0], S->tb.ss.root, S->d_rec);
  SCU_F(cudaMemcpyAsync(B.h_rec, S->d_rec, nc * sizeof(SRecord), cudaMemcpyDeviceToHost, S->cs));
  SCU_F(cudaMemcpyAsync(B.h_err, S->d_err, 8, cudaMemcpyDeviceToHost, S->cs));
  SCU_F(cudaMemcpyAsync(B.h_counters, S->tb.counters, 16, cudaMemcpyDeviceToHost, S->cs));
  SCU_F(cudaEventRecord(B.done, S->cs));
  return RV_OK;
}

// wait for batch b and turn its device status into the chunks' status
rv_status finish_batch(rv_service* S, InFlight& b) {
  if (b.launch != RV_OK) {
    cudaStreamSynchronize(S->cs);               // nothing of it may still run when its buffer is reused
    return b.launch;
  }
  const Buf& B = S->buf[b.buf];
  SCU_F(cudaEventSynchronize(B.done));
  const unsigned e = B.h_err[0] | B.h_err[1];
  if (e & ERR_LETTER) return rv_fail(RV_EINVAL, "predicate code out of range in a streamed chunk");
  if (e & ERR_TABLE) return rv_fail(RV_ENOMEM, "binding table full");
  if (e & ERR_SPIN) return rv_fail(RV_ETIMEOUT, "a bounded device wait gave up");
  if (e) return rv_fail(RV_EINTERNAL, "device status 0x%x", e);
  return RV_OK;
}

// A closed stream's device state (its table entries, its root counts) is
// cleared by kernels queued on the kernel stream once none of its chunks is in
// a launched, unpublished batch -- so after every batch that carried them --
// and its slot is given back when those kernels have run.
struct Retiring {
  std::vector<rv_stream*> streams;
  cudaEvent_t done = nullptr;
};

bool retirable(rv_service* S) {
  for (rv_stream* st : S->to_retire)
    if (st->in_flight == 0) return true;
  return false;
}

rv_status launch_retire(rv_service* S, std::vector<Retiring>& retiring) {
  Retiring r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->to_retire.begin(); it != S->to_retire.end();) {
      if ((*it)->in_flight == 0) { r.streams.push_back(*it); it = S->to_retire.erase(it); }
      else ++it;
    }
  }
  if (r.streams.empty()) return RV_OK;
  for (rv_stream* st : r.streams) {
    RV_LAUNCH("k_s_retire", k_s_retire, 1024, 256, 0, S->cs, S->tb.bind, S->bcap, st->id, S->tb.bind_cap_ids,
              (int*)&S->tb.counters[2], S->tb.free_bind, S->tb.ss.root);
    if (S->f.n_quant == 2)
      RV_LAUNCH("k_s_retire", k_s_retire, 1024, 256, 0, S->cs, S->tb.outer, S->ocap, st->id, S->tb.outer_cap_ids,
                (int*)&S->tb.counters[3], S->tb.free_outer, (unsigned long long*)nullptr);
  }
  SCU_F(cudaGetLastError());
  SCU_F(cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
  SCU_F(cudaMemcpyAsync(S->h_retire_counters, S->tb.counters, 16, cudaMemcpyDeviceToHost, S->cs));
  SCU_F(cudaEventRecord(r.done, S->cs));
  retiring.push_back(std::move(r));
  return RV_OK;
}

// give back the slots of retirements whose kernels have run (waiting for
// them when `block`)
rv_status poll_retire(rv_service* S, std::vector<Retiring>& retiring, bool block) {
  while (!retiring.empty()) {
    Retiring& r = retiring.front();
    cudaError_t e = block ? cudaEventSynchronize(r.done) : cudaEventQuery(r.done);
    if (e == cudaErrorNotReady) return RV_OK;
    cudaEventDestroy(r.done);
    if (e != cudaSuccess) return rv_fail(RV_ECUDA, "retire: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(S->mu);
    const unsigned int* hc = S->h_retire_counters;
    if (retiring.size() == 1) {     // the latest copy of the counters: the admission figures
      S->bindings_used = hc[0] - (uint64_t)std::max(0, (int)hc[2]);
      S->outer_used = hc[1] - (uint64_t)std::max(0, (int)hc[3]);
    }
    for (rv_stream* st : r.streams) {
      S->slots[st->id] = nullptr;
      S->free_slots.push_back(st->id);
      S->retired += 1;
      delete st;
    }
    retiring.erase(retiring.begin());
    S->cv_work.notify_all();
  }
  return RV_OK;
}

// take the next batch: at most one chunk per stream (each chunk's verdict is
// that of exactly its stream's prefix), up to max_batch_events
void take_batch(rv_service* S, std::vector<Staged>& batch) {
  uint64_t total = 0;
  std::vector<char> taken(S->slots.size(), 0);
  for (auto it = S->pending.begin(); it != S->pending.end();) {
    const uint32_t sid = it->stream;
    if (taken[sid] || total + it->n > S->cfg.max_batch_events) { ++it; continue; }
    taken[sid] = 1;
    it->st->in_flight += 1;
    total += it->n;
    batch.push_back(std::move(*it));
    it = S->pending.erase(it);
  }
}

void worker_main(rv_service* S) {
  cudaSetDevice(S->device);
  InFlight prev;
  bool have_prev = false;
  int next_buf = 0;
  std::vector<Retiring> retiring;
  auto fail = [&](rv_status st) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = st;
    S->cv_out.notify_all();
  };
  while (true) {
    InFlight cur;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (!have_prev && retiring.empty())
        S->cv_work.wait(lk, [&] {
          return S->stop || (S->fatal == RV_OK && (!S->pending.empty() || retirable(S)));
        });
      if (S->stop && !have_prev && (S->pending.empty() || S->fatal != RV_OK)) break;
      if (S->fatal == RV_OK) take_batch(S, cur.batch);
    }
    if (!cur.batch.empty()) {
      cur.buf = next_buf;
      next_buf ^= 1;
      cur.launch = launch_batch(S, cur);     // its copies overlap the previous batch's kernels
    }
    if (have_prev) {
      const rv_status st = finish_batch(S, prev);
      publish(S, prev, st, Clock::now());
      have_prev = false;
    }
    if (!cur.batch.empty()) {
      prev = std::move(cur);
      have_prev = true;
    }
    if (S->fatal == RV_OK) {
      rv_status st = launch_retire(S, retiring);
      if (st == RV_OK) st = poll_retire(S, retiring, !have_prev);
      if (st != RV_OK) fail(st);
    }
  }
  for (Retiring& r : retiring) { cudaEventSynchronize(r.done); cudaEventDestroy(r.done); }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

void free_bufs(rv_service* S) {
  for (Buf& B : S->buf) {
    if (B.h_keys) cudaFreeHost(B.h_keys);
    if (B.h_pred) cudaFreeHost(B.h_pred);
    if (B.h_chunks) cudaFreeHost(B.h_chunks);
    if (B.h_rec) cudaFreeHost(B.h_rec);
    if (B.h_err) cudaFreeHost(B.h_err);
    if (B.h_counters) cudaFreeHost(B.h_counters);
    if (B.copied) cudaEventDestroy(B.copied);
    if (B.done) cudaEventDestroy(B.done);
    B = Buf{};
  }
}

}  // namespace

extern "C" rv_status rv_service_open(const rv_formula* f, const rv_service_cfg* cfg, rv_service** out) {
  if (!f || !out) return rv_fail(RV_EINVAL, "null argument");
  *out = nullptr;
  if (f->n_quant < 1 || f->n_quant > 2) return rv_fail(RV_EUNSUPPORTED, "streaming needs one or two quantifiers");
  if (f->n_quant == 1 && f->key_bits != 32) return rv_fail(RV_EUNSUPPORTED, "one-quantifier streams use 32-bit keys");
  if (f->n_cmp) return rv_fail(RV_EUNSUPPORTED, "streams carry no value column: no comparison atoms");
  rv_service* S = new (std::nothrow) rv_service();
  if (!S) return rv_fail(RV_ENOMEM, "out of host memory");
  S->f = *f;
  rv_service_cfg c = cfg ? *cfg : rv_service_cfg{};
  if (!c.max_bindings) c.max_bindings = 1 << 24;
  if (!c.max_outer) c.max_outer = f->n_quant == 2 ? (1 << 22) : 1;
  if (!c.max_batch_events) c.max_batch_events = 1 << 22;
  if (!c.max_staged_events) c.max_staged_events = 1 << 25;
  if (!c.max_streams) c.max_streams = 64;
  if (c.max_streams > 65535 || c.max_bindings > 0x7FFFFF00ull || c.max_outer > 0x7FFFFF00ull)
    return delete S, rv_fail(RV_EINVAL, "service limits out of range");
  S->cfg = c;
  S->key_bytes = f->key_bits / 8;
  cudaGetDevice(&S->device);
  S->bcap = pow2_at_least(c.max_bindings * 2);
  S->ocap = pow2_at_least(c.max_outer * 2);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = a256(off + bytes); return r; };
  const size_t o_bind = take(S->bcap * sizeof(Entry)), o_outer = take(S->ocap * sizeof(Entry));
  const size_t o_fb = take(c.max_bindings * 4), o_fo = take(c.max_outer * 4);
  const size_t o_bstate = take(c.max_bindings), o_bverd = take(c.max_bindings), o_bstream = take(c.max_bindings * 2);
  const size_t o_ocnt = take(c.max_outer * 24), o_overd = take(c.max_outer), o_ostream = take(c.max_outer * 2);
  const size_t o_root = take((size_t)c.max_streams * 6 * 8), o_ctr = take(16);
  size_t o_keys[2], o_pred[2], o_chunks[2];
  for (int i = 0; i < 2; ++i) {
    o_keys[i] = take(c.max_batch_events * S->key_bytes);
    o_pred[i] = take(c.max_batch_events);
    o_chunks[i] = take((size_t)c.max_streams * sizeof(ChunkDesc));
  }
  const size_t o_ids = take(c.max_batch_events * 8);
  const size_t o_rec = take((size_t)c.max_streams * sizeof(SRecord)), o_err = take(16);
  S->ws_bytes = rv_offline_stream_ws(f, c.max_batch_events);
  const size_t o_ws = take(S->ws_bytes);
  S->dmem = rv_dev_alloc(off);
  if (!S->dmem) { delete S; return rv_fail(RV_ENOMEM, "cannot allocate %zu bytes of service memory", off); }
  unsigned char* D = (unsigned char*)S->dmem;
  S->tb.bind = (Entry*)(D + o_bind);
  S->tb.outer = (Entry*)(D + o_outer);
  S->tb.bind_mask = S->bcap - 1;
  S->tb.outer_mask = S->ocap - 1;
  S->tb.bind_cap_ids = (uint32_t)c.max_bindings;
  S->tb.outer_cap_ids = (uint32_t)c.max_outer;
  S->tb.counters = (unsigned int*)(D + o_ctr);
  S->tb.free_bind = (uint32_t*)(D + o_fb);
  S->tb.free_outer = (uint32_t*)(D + o_fo);
  S->tb.ss.bstate = D + o_bstate;
  S->tb.ss.bverdict = D + o_bverd;
  S->tb.ss.bstream = (uint16_t*)(D + o_bstream);
  S->tb.ss.ocounts = (uint32_t*)(D + o_ocnt);
  S->tb.ss.overdict = D + o_overd;
  S->tb.ss.ostream = (uint16_t*)(D + o_ostream);
  S->tb.ss.root = (unsigned long long*)(D + o_root);
  for (int i = 0; i < 2; ++i) {
    S->buf[i].d_keys = D + o_keys[i];
    S->buf[i].d_pred = D + o_pred[i];
    S->buf[i].d_chunks = (ChunkDesc*)(D + o_chunks[i]);
  }
  S->d_ids = (uint64_t*)(D + o_ids);
  S->d_rec = (SRecord*)(D + o_rec);
  S->d_err = (unsigned int*)(D + o_err);
  S->ws = D + o_ws;
  S->slots.assign(c.max_streams, nullptr);
  for (int i = c.max_streams - 1; i >= 0; --i) S->free_slots.push_back((uint32_t)i);
  auto fail = [&](rv_status s2) { rv_service_close(S); return s2; };
  if (cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->cp, cudaStreamNonBlocking) != cudaSuccess)
    return fail(rv_fail(RV_ECUDA, "stream"));
  for (Buf& B : S->buf) {
    if (cudaMallocHost(&B.h_keys, c.max_batch_events * S->key_bytes) != cudaSuccess ||
        cudaMallocHost(&B.h_pred, c.max_batch_events) != cudaSuccess ||
        cudaMallocHost(&B.h_chunks, (size_t)c.max_streams * sizeof(ChunkDesc)) != cudaSuccess ||
        cudaMallocHost(&B.h_rec, (size_t)c.max_streams * sizeof(SRecord)) != cudaSuccess ||
        cudaMallocHost(&B.h_err, 16) != cudaSuccess || cudaMallocHost(&B.h_counters, 16) != cudaSuccess)
      return fail(rv_fail(RV_ENOMEM, "cannot allocate pinned staging"));
    memset(B.h_counters, 0, 16);
    if (cudaEventCreateWithFlags(&B.copied, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming) != cudaSuccess)
      return fail(rv_fail(RV_ECUDA, "event"));
  }
  if (cudaMallocHost(&S->h_retire_counters, 16) != cudaSuccess)
    return fail(rv_fail(RV_ENOMEM, "cannot allocate pinned staging"));
  k_s_init<<<1024, 256, 0, S->cs>>>(S->tb.bind, S->bcap);
  k_s_init<<<1024, 256, 0, S->cs>>>(S->tb.outer, S->ocap);
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
  for (rv_stream* st : S->slots) delete st;     // closed, unretired streams still hold their slot
  if (S->h_retire_counters) cudaFreeHost(S->h_retire_counters);
  if (S->cs) { cudaStreamSynchronize(S->cs); cudaStreamDestroy(S->cs); }
  if (S->cp) { cudaStreamSynchronize(S->cp); cudaStreamDestroy(S->cp); }
  free_bufs(S);
  if (S->dmem) rv_dev_free(S->dmem);
  delete S;
  return RV_OK;
}

extern "C" rv_status rv_stream_open(rv_service* S, rv_stream** out) {
  if (!S || !out) return rv_fail(RV_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->fatal != RV_OK) return rv_fail(S->fatal, "service failed earlier");
  if (S->free_slots.empty())
    return rv_fail(RV_EAGAIN, "all %d stream slots are in use or being retired", S->cfg.max_streams);
  rv_stream* st = new (std::nothrow) rv_stream();
  if (!st) return rv_fail(RV_ENOMEM, "out of host memory");
  st->svc = S;
  st->id = S->free_slots.back();
  S->free_slots.pop_back();
  S->slots[st->id] = st;
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
    if (S->fatal != RV_OK) return rv_fail(S->fatal, "service failed earlier");
    if (st->failed) return rv_fail(RV_EINVAL, "an earlier chunk of this stream failed on the device; close it");
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
    if (st->closed) {                 // closed while the chunk was copied: drop it
      S->staged_events -= sc.n;
      S->reserved_bindings -= sc.n;
      return rv_fail(RV_EINVAL, "stream is closed");
    }
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
  if (st->closed) return rv_fail(RV_EINVAL, "stream is closed");
  auto ready = [&] { return !st->out.empty() || S->fatal != RV_OK; };
  if (!ready() && timeout_us > 0)
    S->cv_out.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
  int k = 0;
  while (k < max && !st->out.empty()) { out[k++] = st->out.front(); st->out.pop_front(); }
  *n = k;
  if (k == 0) {
    if (S->fatal != RV_OK) return rv_fail(S->fatal, "service failed");
    return rv_fail(RV_ETIMEOUT, "no verdict within %d us", timeout_us);
  }
  return RV_OK;
}

extern "C" rv_status rv_stream_close(rv_stream* st) {
  if (!st) return RV_OK;
  rv_service* S = st->svc;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (st->closed) return RV_OK;
    st->closed = true;
    st->out.clear();
    for (auto it = S->pending.begin(); it != S->pending.end();) {   // drop its queued chunks
      if (it->st == st) {
        S->staged_events -= it->n;
        S->reserved_bindings -= it->n;
        it = S->pending.erase(it);
      } else {
        ++it;
      }
    }
    S->to_retire.push_back(st);
  }
  S->cv_work.notify_all();
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
