// serve.cu -- continuous-batching server for factor+solve requests.
//
// Requests (LU + Rgetrs or Cholesky + Rpotrs, host matrices) are admitted in
// arrival order while their device state fits the memory budget; admitted
// matrices, pivots and right-hand sides stay resident on the device until the
// request completes.  Two lanes run concurrently on their own streams:
//   small lane  n <= small_n_max: every admitted, not yet started request is
//               put into the next persistent batched launch as soon as the
//               previous small launch has finished (continuous batching);
//   large lanes n >  small_n_max: through the blocked multi-SM routines, one
//               request per lane, large_lanes lanes (streams) at once.
// The caller drives the server: posit_serve_poll retires finished launches
// (CUDA events, no blocking), frees their memory, admits waiting requests
// and starts launches.  Results are bit-identical to the single-request
// routines, alone or in any mix.
#include <algorithm>
#include <deque>
#include <new>
#include <vector>

#include "internal.cuh"

namespace posit {
namespace {

struct Req {
  posit_request r;
  size_t bytes;
  char *dev;  // one allocation: A | B | ipiv | info
  uint32_t *dA, *dB;
  int32_t *dipiv, *dinfo;
};

struct Launch {
  cudaEvent_t done;
  std::vector<int> reqs;
  void *desc;  // device descriptor array (small lane), freed on completion
  int lane;    // -1: small lane, else the large lane index
};

struct Lane {
  cudaStream_t stream = nullptr;
  void *scratch = nullptr;
  bool busy = false;
};

}  // namespace
}  // namespace posit

struct posit_server {
  posit_serve_config cfg;
  cudaStream_t s_small = nullptr, s_copy = nullptr;
  std::vector<posit::Lane> lanes;  // large lanes
  std::vector<posit::Req> reqs;
  std::vector<int> free_slots;
  std::deque<int> pending, small_ready, large_ready;
  std::vector<posit::Launch> inflight;
  bool small_busy = false;
  size_t used = 0;
  size_t lane_scratch = 0;  // bytes of each large lane's scratch
  void *ws = nullptr;  // batched workspace (small lane)
  posit_problem *stage = nullptr;  // pinned staging for descriptors
  int64_t stage_cap = 0;
  int64_t admitted = 0, completed = 0, launches = 0, batched = 0, largest = 0;
};

namespace posit {
namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t req_bytes(const posit_request &r) {
  size_t n = (size_t)r.n, k = (size_t)r.nrhs;
  return align256(n * n * 4) + align256(n * k * 4) + align256(n * 4) + 256;
}

int admit(posit_server *sv, int id) {
  Req &q = sv->reqs[id];
  void *p = nullptr;
  if (cudaMallocAsync(&p, q.bytes, sv->s_copy) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  const size_t n = (size_t)q.r.n, k = (size_t)q.r.nrhs;
  q.dev = static_cast<char *>(p);
  q.dA = reinterpret_cast<uint32_t *>(q.dev);
  q.dB = reinterpret_cast<uint32_t *>(q.dev + align256(n * n * 4));
  q.dipiv = reinterpret_cast<int32_t *>(q.dev + align256(n * n * 4) + align256(n * k * 4));
  q.dinfo = reinterpret_cast<int32_t *>(q.dev + align256(n * n * 4) + align256(n * k * 4) +
                                        align256(n * 4));
  if (cudaMemcpyAsync(q.dA, q.r.A, n * n * 4, cudaMemcpyHostToDevice, sv->s_copy) != cudaSuccess ||
      cudaMemcpyAsync(q.dB, q.r.B, n * k * 4, cudaMemcpyHostToDevice, sv->s_copy) != cudaSuccess ||
      cudaMemsetAsync(q.dinfo, 0, 4, sv->s_copy) != cudaSuccess)
    return POSIT_ERR_CUDA;
  sv->used += q.bytes;
  sv->admitted++;
  return POSIT_OK;
}

int finish_copies(posit_server *sv, const Req &q, cudaStream_t s) {
  const size_t n = (size_t)q.r.n, k = (size_t)q.r.nrhs;
  if (cudaMemcpyAsync(q.r.X, q.dB, n * k * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(q.r.info, q.dinfo, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return POSIT_ERR_CUDA;
  (void)sv;
  return POSIT_OK;
}

int start_small(posit_server *sv, cudaEvent_t ready) {
  const int64_t cnt = std::min<int64_t>((int64_t)sv->small_ready.size(), sv->cfg.max_batch);
  if (cnt <= 0) return POSIT_OK;
  Launch L;
  L.lane = -1;
  int max_n = 0, max_k = 0;
  for (int64_t i = 0; i < cnt; ++i) {
    int id = sv->small_ready.front();
    sv->small_ready.pop_front();
    L.reqs.push_back(id);
    const Req &q = sv->reqs[id];
    posit_problem &d = sv->stage[i];
    d.kind = q.r.kind; d.n = q.r.n; d.nrhs = q.r.nrhs; d.reserved = 0;
    d.lda = q.r.n; d.ldb = q.r.n;
    d.A = q.dA; d.B = q.dB; d.ipiv = q.dipiv; d.info = q.dinfo;
    max_n = std::max(max_n, q.r.n);
    max_k = std::max(max_k, q.r.nrhs);
  }
  if (cudaStreamWaitEvent(sv->s_small, ready, 0) != cudaSuccess) return POSIT_ERR_CUDA;
  if (cudaMallocAsync(&L.desc, cnt * sizeof(posit_problem), sv->s_small) != cudaSuccess) {
    cudaGetLastError();
    return POSIT_ERR_ALLOC;
  }
  if (cudaMemcpyAsync(L.desc, sv->stage, cnt * sizeof(posit_problem), cudaMemcpyHostToDevice,
                      sv->s_small) != cudaSuccess)
    return POSIT_ERR_CUDA;
  // the staging buffer is reused by the next launch only after this one has
  // completed (the small lane runs one launch at a time)
  int st = batched_launch(static_cast<posit_problem *>(L.desc), nullptr, cnt,
                          sv->cfg.small_n_max, sv->cfg.max_nrhs, sv->cfg.plan, sv->ws,
                          sv->s_small);
  if (st) return st;
  for (int id : L.reqs)
    if ((st = finish_copies(sv, sv->reqs[id], sv->s_small))) return st;
  if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(L.done, sv->s_small) != cudaSuccess)
    return POSIT_ERR_CUDA;
  sv->inflight.push_back(L);
  sv->small_busy = true;
  sv->launches++;
  sv->batched += cnt;
  sv->largest = std::max(sv->largest, cnt);
  return POSIT_OK;
}

int start_large(posit_server *sv, int lane, cudaEvent_t ready) {
  if (sv->large_ready.empty()) return POSIT_OK;
  int id = sv->large_ready.front();
  sv->large_ready.pop_front();
  const Req &q = sv->reqs[id];
  Lane &ln = sv->lanes[lane];
  if (cudaStreamWaitEvent(ln.stream, ready, 0) != cudaSuccess) return POSIT_ERR_CUDA;
  int st;
  const int64_t n = q.r.n, k = q.r.nrhs;
  if (q.r.kind == POSIT_LU) {
    st = getrf_run(n, n, q.dA, n, q.dipiv, q.dinfo, ln.scratch, ln.stream);
    if (!st)
      st = getrs_run(false, n, k, q.dA, n, q.dipiv, q.dB, n, ln.scratch, sv->lane_scratch,
                     ln.stream);
  } else {
    const bool upper = q.r.kind == POSIT_CHOLESKY_U;
    st = potrf_run(upper, n, q.dA, n, q.dinfo, ln.scratch, ln.stream);
    // the solve is skipped on the device when info != 0 (B then keeps b)
    if (!st)
      st = potrs_run_guarded(upper, n, k, q.dA, n, q.dB, n, q.dinfo, ln.scratch,
                             sv->lane_scratch, ln.stream);
  }
  if (st) return st;
  if ((st = finish_copies(sv, q, ln.stream))) return st;
  Launch L;
  L.lane = lane;
  L.desc = nullptr;
  L.reqs.push_back(id);
  if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(L.done, ln.stream) != cudaSuccess)
    return POSIT_ERR_CUDA;
  sv->inflight.push_back(L);
  ln.busy = true;
  sv->launches++;
  return POSIT_OK;
}

}  // namespace
}  // namespace posit

using namespace posit;

extern "C" int posit_serve_open(const posit_serve_config *cfg, posit_server **out) {
  if (!cfg) return -1;
  if (!out) return -2;
  if (cfg->budget_bytes <= 0 || cfg->small_n_max < 1 || cfg->small_n_max > 46340 ||
      cfg->max_batch < 1 || cfg->max_nrhs < 1 || cfg->large_lanes < 0 || cfg->large_lanes > 64 ||
      cfg->batch_only_n_max < 0)
    return -1;
  posit_server *sv = new (std::nothrow) posit_server();
  if (!sv) return POSIT_ERR_ALLOC;
  sv->cfg = *cfg;
  if (sv->cfg.large_lanes == 0) sv->cfg.large_lanes = 16;
  int st = POSIT_OK;
  if (cudaStreamCreateWithFlags(&sv->s_small, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->s_copy, cudaStreamNonBlocking) != cudaSuccess)
    st = POSIT_ERR_CUDA;
  size_t wsb = batched_workspace_bytes(cfg->small_n_max, cfg->max_nrhs, cfg->plan);
  // solves of any n fit (fewer right-hand sides per launch past n = 2^20)
  size_t scr = std::max(getrf_scratch_bytes(), solve_scratch_bytes(1 << 20));
  sv->lane_scratch = scr;
  if (!st && (!wsb || cudaMalloc(&sv->ws, wsb) != cudaSuccess)) st = POSIT_ERR_ALLOC;
  sv->lanes.resize(sv->cfg.large_lanes);
  for (auto &ln : sv->lanes) {
    if (st) break;
    if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess)
      st = POSIT_ERR_CUDA;
    else if (cudaMalloc(&ln.scratch, scr) != cudaSuccess)
      st = POSIT_ERR_ALLOC;
  }
  sv->stage_cap = cfg->max_batch;
  if (!st && cudaMallocHost(&sv->stage, sizeof(posit_problem) * cfg->max_batch) != cudaSuccess)
    st = POSIT_ERR_ALLOC;
  if (st) {
    cudaGetLastError();
    posit_serve_close(sv);
    return st;
  }
  *out = sv;
  return POSIT_OK;
}

extern "C" int posit_serve_submit(posit_server *sv, const posit_request *req) {
  if (!sv) return -1;
  if (!req || (req->kind != POSIT_LU && req->kind != POSIT_CHOLESKY &&
               req->kind != POSIT_CHOLESKY_U) || req->n < 1 ||
      req->nrhs < 1 || req->nrhs > sv->cfg.max_nrhs || !req->A || !req->B || !req->X || !req->info)
    return -2;
  posit::Req q;
  q.r = *req;
  q.bytes = posit::req_bytes(*req);
  if (q.bytes > (size_t)sv->cfg.budget_bytes) return -2;
  q.dev = nullptr;
  int id;
  if (!sv->free_slots.empty()) {
    id = sv->free_slots.back();
    sv->free_slots.pop_back();
    sv->reqs[id] = q;
  } else {
    id = (int)sv->reqs.size();
    sv->reqs.push_back(q);
  }
  sv->pending.push_back(id);
  return POSIT_OK;
}

extern "C" int posit_serve_poll(posit_server *sv, uint64_t *done_tags, int64_t max_done,
                                int64_t *n_done) {
  if (!sv) return -1;
  if (max_done < 0 || (max_done > 0 && !done_tags)) return -3;
  if (!n_done) return -4;
  *n_done = 0;
  // 1. retire finished launches (in any order), up to max_done requests
  for (size_t i = 0; i < sv->inflight.size();) {
    Launch &L = sv->inflight[i];
    if ((int64_t)(*n_done + L.reqs.size()) > max_done) { ++i; continue; }
    cudaError_t e = cudaEventQuery(L.done);
    if (e == cudaErrorNotReady) { ++i; continue; }
    if (e != cudaSuccess) return POSIT_ERR_CUDA;
    cudaEventDestroy(L.done);
    cudaStream_t ls = L.lane < 0 ? sv->s_small : sv->lanes[L.lane].stream;
    for (int id : L.reqs) {
      Req &q = sv->reqs[id];
      cudaFreeAsync(q.dev, ls);
      sv->used -= q.bytes;
      done_tags[(*n_done)++] = q.r.tag;
      sv->free_slots.push_back(id);
      sv->completed++;
    }
    if (L.desc) cudaFreeAsync(L.desc, sv->s_small);
    if (L.lane < 0) sv->small_busy = false; else sv->lanes[L.lane].busy = false;
    sv->inflight.erase(sv->inflight.begin() + i);
  }
  // 2. admit waiting requests in arrival order while they fit the budget
  bool any = false;
  while (!sv->pending.empty()) {
    int id = sv->pending.front();
    if (sv->used + sv->reqs[id].bytes > (size_t)sv->cfg.budget_bytes) break;
    int st = admit(sv, id);
    if (st) return st;
    sv->pending.pop_front();
    if (sv->reqs[id].r.n <= sv->cfg.small_n_max) sv->small_ready.push_back(id);
    else sv->large_ready.push_back(id);
    any = true;
  }
  // 3. start launches on idle lanes; they wait for the admitted copies
  (void)any;
  int idle = 0;
  for (auto &ln : sv->lanes) idle += !ln.busy;
  // latency first: idle large lanes left over after the large requests take
  // the waiting small requests that are too big to be quick in one CTA
  {
    int spare = idle - (int)sv->large_ready.size();
    for (auto it = sv->small_ready.begin(); spare > 0 && it != sv->small_ready.end();) {
      if (sv->reqs[*it].r.n > sv->cfg.batch_only_n_max) {
        sv->large_ready.push_back(*it);
        it = sv->small_ready.erase(it);
        --spare;
      } else {
        ++it;
      }
    }
  }
  bool small_go = !sv->small_busy && !sv->small_ready.empty();
  bool large_go = idle > 0 && !sv->large_ready.empty();
  if (small_go || large_go) {
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, sv->s_copy) != cudaSuccess)
      return POSIT_ERR_CUDA;
    int st = POSIT_OK;
    if (small_go) st = start_small(sv, ready);
    for (size_t l = 0; !st && l < sv->lanes.size() && !sv->large_ready.empty(); ++l)
      if (!sv->lanes[l].busy) st = start_large(sv, (int)l, ready);
    cudaEventDestroy(ready);
    if (st) return st;
  }
  return POSIT_OK;
}

extern "C" int posit_serve_stats(const posit_server *sv, posit_serve_stats_t *st) {
  if (!sv) return -1;
  if (!st) return -2;
  st->pending = (int64_t)sv->pending.size();
  st->admitted = sv->admitted;
  st->completed = sv->completed;
  st->inflight_launches = (int64_t)sv->inflight.size();
  st->launches = sv->launches;
  st->device_bytes_in_use = (int64_t)sv->used;
  st->batched_requests = sv->batched;
  st->largest_batch = sv->largest;
  return POSIT_OK;
}

extern "C" int posit_serve_close(posit_server *sv) {
  if (!sv) return -1;
  if (sv->s_small) cudaStreamSynchronize(sv->s_small);
  for (auto &ln : sv->lanes)
    if (ln.stream) cudaStreamSynchronize(ln.stream);
  if (sv->s_copy) cudaStreamSynchronize(sv->s_copy);
  for (auto &L : sv->inflight) {
    cudaEventDestroy(L.done);
    if (L.desc) cudaFree(L.desc);
    for (int id : L.reqs) cudaFree(sv->reqs[id].dev);
  }
  for (int id : sv->small_ready) cudaFree(sv->reqs[id].dev);
  for (int id : sv->large_ready) cudaFree(sv->reqs[id].dev);
  if (sv->ws) cudaFree(sv->ws);
  for (auto &ln : sv->lanes) {
    if (ln.scratch) cudaFree(ln.scratch);
    if (ln.stream) cudaStreamDestroy(ln.stream);
  }
  if (sv->stage) cudaFreeHost(sv->stage);
  if (sv->s_small) cudaStreamDestroy(sv->s_small);
  if (sv->s_copy) cudaStreamDestroy(sv->s_copy);
  delete sv;
  return POSIT_OK;
}
