// Serving loop: chemistry sub-steps requested by many concurrent flow solvers.
//
// In the paper one solver owns the GPU and its time loop calls the chemistry step once per CFD
// step (§3.1, Fig. 1); here many solvers share one GPU.  Each solver registers its state arrays
// once (they stay resident on the device) and then submits one request per sub-step.  A server
// thread
//   * admits queued requests in arrival order, skipping ahead to requests that fit, while the
//     resident states plus the workspace of the requests in flight stay within the device-memory
//     budget, and at most one request per state is in flight;
//   * batches the admitted FP64 requests of each mechanism into one job of the persistent
//     integrator (their cells share one work queue), surrogate requests into their own launches,
//     each on the next free stream of a small pool so that launches overlap on the device;
//   * runs an FP64 job as time slices: every slice stops claiming cells after slice_ms, the
//     server reads the queue counter back and re-issues the slice until the queue is drained.
//     Cells are claimed in queue order, so the claimed part is a prefix of the queue and a request
//     is complete as soon as the counter passes its last chunk.  Between slices the other streams'
//     launches get the SMs: a small request is not stuck behind a persistent launch that would
//     otherwise hold every SM for seconds;
//   * retires requests when their launch or slice completes, records the latency from submission
//     to completion and frees their budget, so requests arriving meanwhile are admitted as slots
//     and memory free up (continuous batching).
// chem_serve_poll never blocks; chem_serve_wait blocks at most the given timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "chem_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3 };

struct StateRec {
  chem_mech_t mech;
  chem_model_t model;
  double* T;
  double* p;
  double* Y;
  int64_t ld, ncells;
  size_t resident;
  bool busy = false;
};

struct Req {
  uint64_t id;
  int state;
  int route;
  double dt, rtol, atol;
  int status = Q_QUEUED;
  size_t bytes = 0;
  Clock::time_point t_submit, t_done;
  std::string error;
};

struct Launch {
  cudaEvent_t ev;
  int stream;
  std::vector<uint64_t> reqs;
  size_t bytes;
  // FP64 job run as time slices: its segments, the queue end of each request's chunks, and how
  // many of its requests (in queue order) have completed
  bool sliced = false;
  chem_mech_t mech = nullptr;
  std::vector<chem_segment> segs;
  std::vector<long long> seg_end;
  long long issued_total = 0;     // queue end the running slice was issued with
  size_t ndone = 0;
  // a job whose slice ended while surrogate passes run waits (at most max_pause) before its next
  // slice, so that the passes' kernels find the SMs free
  bool paused = false;
  Clock::time_point paused_since;
};

}  // namespace

extern "C" int chem_surrogate_advance_batch(chem_model_t md, chem_mech_t mech, const chem_segment* segs,
                                            int nseg, chem_stream_t stream);

struct chem_server_s {
  size_t budget = 0, resident = 0, inflight = 0;
  int device = 0;
  std::vector<cudaStream_t> streams;   // [0, n_fp64): FP64 jobs; the rest: surrogate launches
  std::vector<bool> stream_busy;
  int n_fp64 = 4;
  std::map<int, StateRec> states;
  int next_state = 1;
  std::map<uint64_t, Req> reqs;
  std::deque<uint64_t> pending;
  uint64_t next_req = 1;
  std::vector<Launch> launches;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  bool stop = false;
  uint64_t n_submitted = 0;                    // submissions so far: the idle server waits for a new one
  int64_t n_launches = 0, n_batched = 0, n_done = 0, n_failed = 0, max_concurrent = 0, n_slices = 0;
  int64_t n_joined = 0;                        // FP64 requests that joined a running time-sliced job
  double idle_poll_us = 20.0;
  unsigned long long slice_ns = 20000000ull;   // 0: FP64 jobs run unsliced
  unsigned long long max_pause_ns = 20000000ull;  // longest wait of an FP64 job for surrogate passes
  unsigned long long* d_counter = nullptr;     // one work-queue counter per stream (device)
  unsigned long long* h_counter = nullptr;     // its read-back copy (pinned host memory)
  unsigned long long* h_reset = nullptr;       // values the counters are set back to (pinned)
  // per stream: a nonzero word ends the stream's running FP64 slice early (device; set when a
  // surrogate pass is issued, so that its kernels need not wait for the slice's time budget)
  unsigned int* d_stop = nullptr;
  unsigned int* h_flags = nullptr;             // {0, 1}: the values copied into d_stop (pinned)
};

// a slice ends early on request only after this long (every slice makes progress)
constexpr unsigned long long kMinSliceNs = 2000000ull;

namespace {

size_t request_bytes(const StateRec& s, int route) {
  if (route == CHEM_ROUTE_SURROGATE)    // gathered state copy; network output, box flags, fallback list
    return (size_t)s.ncells * (((size_t)s.mech->ns + 2) * 8 + 1 + (size_t)s.mech->ns * 4 + 1 + 4) + 4096;
  return 4096;                           // work-queue counter
}

// the key surrogate requests are batched by: one gathered pass needs one model, mechanism, step
// and tolerance pair
struct SurKey {
  chem_model_t model;
  chem_mech_t mech;
  double dt, rtol, atol;
  bool operator<(const SurKey& o) const {
    if (model != o.model) return model < o.model;
    if (mech != o.mech) return mech < o.mech;
    if (dt != o.dt) return dt < o.dt;
    if (rtol != o.rtol) return rtol < o.rtol;
    return atol < o.atol;
  }
};

void server_loop(chem_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    const uint64_t submitted = S->n_submitted;
    // ---- retire finished launches ----
    bool progressed = false;
    bool sur_running = false;
    for (const Launch& L : S->launches)
      if (!L.sliced && cudaEventQuery(L.ev) == cudaErrorNotReady) sur_running = true;
    for (size_t i = 0; i < S->launches.size();) {
      Launch& L = S->launches[i];
      cudaError_t q = cudaEventQuery(L.ev);
      if (q == cudaErrorNotReady) { ++i; continue; }
      const Clock::time_point now = Clock::now();
      if (q == cudaSuccess && L.sliced) {
        // the slice processed every chunk it claimed below the queue end it was issued with;
        // groups that found the queue empty still advanced the counter past that end
        const long long total = L.seg_end.back();
        const long long claimed = (long long)S->h_counter[L.stream];
        const long long done = std::min<long long>(claimed, L.issued_total);
        while (L.ndone < L.reqs.size() && L.seg_end[L.ndone] <= done) {
          Req& r = S->reqs[L.reqs[L.ndone]];
          r.status = Q_DONE;
          r.t_done = now;
          S->states[r.state].busy = false;
          ++S->n_done;
          ++L.ndone;
          progressed = true;
        }
        if (done < total && sur_running && S->max_pause_ns > 0 &&
            (!L.paused || (unsigned long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
                              now - L.paused_since).count() < S->max_pause_ns)) {
          // surrogate passes are running: their kernels get the whole GPU before this job's next
          // slice (requests wait for a pass, not for FP64 slices between its kernels)
          if (!L.paused) { L.paused = true; L.paused_since = now; }
          ++i;
          continue;
        }
        L.paused = false;
        if (done < total) {
          // next slice of the same job, continuing the same queue; requests that joined since the
          // last slice extend it, and a counter that overshot the old end is set back to it
          cudaStream_t strm = S->streams[L.stream];
          int rc = CHEM_OK;
          if (cudaMemcpyAsync(S->d_stop + L.stream, S->h_flags, sizeof(unsigned int), cudaMemcpyHostToDevice,
                              strm) != cudaSuccess)
            rc = chem::cuda_fail(cudaGetLastError(), "cudaMemcpyAsync(server stop flag)");
          if (rc == CHEM_OK && claimed > L.issued_total) {
            S->h_reset[L.stream] = (unsigned long long)L.issued_total;
            if (cudaMemcpyAsync(S->d_counter + L.stream, S->h_reset + L.stream, sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, strm) != cudaSuccess)
              rc = chem::cuda_fail(cudaGetLastError(), "cudaMemcpyAsync(server counter)");
          }
          if (rc == CHEM_OK)
            rc = chem::launch_advance_slice(L.mech, L.segs.data(), (int)L.segs.size(), S->slice_ns,
                                            S->d_counter + L.stream, nullptr, strm, S->d_stop + L.stream,
                                            kMinSliceNs);
          L.issued_total = total;
          if (rc == CHEM_OK &&
              cudaMemcpyAsync(S->h_counter + L.stream, S->d_counter + L.stream, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, strm) == cudaSuccess &&
              cudaEventRecord(L.ev, strm) == cudaSuccess) {
            ++S->n_slices;
            ++i;
            continue;
          }
          q = cudaErrorLaunchFailure;    // the job's remaining requests fail below
        }
      }
      const std::string err = q == cudaErrorLaunchFailure && L.sliced ? std::string(chem_last_error())
                                                                      : std::string(cudaGetErrorString(q));
      for (size_t k = L.sliced ? L.ndone : 0; k < L.reqs.size(); ++k) {
        const uint64_t id = L.reqs[k];
        Req& r = S->reqs[id];
        r.status = q == cudaSuccess ? Q_DONE : Q_FAILED;
        if (q != cudaSuccess) r.error = err;
        r.t_done = now;
        S->states[r.state].busy = false;
        if (r.status == Q_DONE) ++S->n_done; else ++S->n_failed;
      }
      S->inflight -= L.bytes;
      S->stream_busy[L.stream] = false;
      cudaEventDestroy(L.ev);
      S->launches.erase(S->launches.begin() + i);
      progressed = true;
    }
    if (progressed) S->cv_done.notify_all();
    if (S->stop && S->launches.empty()) break;

    // ---- admit and launch ----
    int free_stream = -1;
    for (size_t k = 0; k < S->streams.size(); ++k)
      if (!S->stream_busy[k]) { free_stream = (int)k; break; }
    if (!S->stop && free_stream >= 0 && !S->pending.empty()) {
      // FP64 requests grouped by mechanism (appended to a running job of that mechanism, else one
      // batched job each) and surrogate requests grouped by model, mechanism, step and tolerances
      // (one gathered pass each)
      std::map<chem_mech_t, std::vector<uint64_t>> fp64;
      std::map<SurKey, std::vector<uint64_t>> sur;
      // states registered while requests run can take resident + inflight past the budget
      size_t avail = S->resident + S->inflight < S->budget ? S->budget - S->resident - S->inflight : 0;
      std::deque<uint64_t> keep;
      for (uint64_t id : S->pending) {
        Req& r = S->reqs[id];
        StateRec& st = S->states[r.state];
        const bool take = !st.busy && r.bytes <= avail;
        if (take) {
          avail -= r.bytes;
          st.busy = true;
          if (r.route == CHEM_ROUTE_FP64) fp64[st.mech].push_back(id);
          else sur[SurKey{st.model, st.mech, r.dt, r.rtol, r.atol}].push_back(id);
        } else {
          keep.push_back(id);
        }
      }
      S->pending.swap(keep);
      // build launches; each needs a free stream, the rest go back to the queue front
      std::vector<std::vector<uint64_t>> groups;
      bool launched = false;             // a group was launched, joined a job or failed: look again right away
      for (auto& kv : fp64) {
        std::vector<uint64_t>& v = kv.second;
        // requests join a running time-sliced job of their mechanism at its next slice boundary:
        // the job's queue grows at its end, so the claimed prefix and the retirement by queue
        // position stay valid (the running slice keeps its own copy of the descriptors)
        size_t used = 0;
        for (Launch& L : S->launches) {
          if (!L.sliced || L.mech != kv.first) continue;
          while (used < v.size() && L.segs.size() < (size_t)chem::kMaxSegsPerLaunch) {
            Req& r = S->reqs[v[used]];
            const StateRec& st = S->states[r.state];
            const long long chunks = chem::advance_queue_chunks(st.mech, st.ncells);
            if (chunks < 0) break;
            chem_segment g{};
            g.T = st.T; g.p = st.p; g.Y = st.Y; g.ld = st.ld; g.ncells = st.ncells;
            g.dt = r.dt; g.rtol = r.rtol; g.atol = r.atol;
            L.segs.push_back(g);
            L.seg_end.push_back(L.seg_end.back() + chunks);
            L.reqs.push_back(r.id);
            L.bytes += r.bytes;
            S->inflight += r.bytes;
            r.status = Q_RUNNING;
            ++S->n_batched;
            ++S->n_joined;
            ++used;
            launched = true;
          }
        }
        // the rest: new jobs of at most kMaxSegsPerLaunch requests each
        for (size_t b = used; b < v.size(); b += chem::kMaxSegsPerLaunch)
          groups.push_back(std::vector<uint64_t>(v.begin() + b, v.begin() + std::min(v.size(), b + chem::kMaxSegsPerLaunch)));
      }
      for (auto& kv : sur) {
        std::vector<uint64_t>& v = kv.second;
        for (size_t b = 0; b < v.size(); b += chem::kMaxSegsPerLaunch)
          groups.push_back(std::vector<uint64_t>(v.begin() + b, v.begin() + std::min(v.size(), b + chem::kMaxSegsPerLaunch)));
      }
      std::vector<uint64_t> back;
      for (auto& grp : groups) {
        // FP64 jobs on the low-priority streams, surrogate launches on the high-priority ones: when
        // a slice's blocks retire, the block scheduler starts a waiting surrogate launch first
        const bool is_fp64 = S->reqs[grp[0]].route == CHEM_ROUTE_FP64;
        int sidx = -1;
        const size_t k0 = is_fp64 ? 0 : (size_t)S->n_fp64, k1 = is_fp64 ? (size_t)S->n_fp64 : S->streams.size();
        for (size_t k = k0; k < k1; ++k)
          if (!S->stream_busy[k]) { sidx = (int)k; break; }
        if (sidx < 0) {
          for (uint64_t id : grp) { S->states[S->reqs[id].state].busy = false; back.push_back(id); }
          continue;
        }
        size_t bytes = 0;
        for (uint64_t id : grp) bytes += S->reqs[id].bytes;
        cudaStream_t strm = S->streams[sidx];
        int rc = CHEM_OK;
        const Req& r0 = S->reqs[grp[0]];
        Launch L;
        if (r0.route == CHEM_ROUTE_FP64) {
          for (uint64_t id : grp) {
            const Req& r = S->reqs[id];
            const StateRec& st = S->states[r.state];
            chem_segment g{};
            g.T = st.T; g.p = st.p; g.Y = st.Y; g.ld = st.ld; g.ncells = st.ncells;
            g.dt = r.dt; g.rtol = r.rtol; g.atol = r.atol;
            L.segs.push_back(g);
          }
          L.sliced = true;
          L.mech = S->states[r0.state].mech;
          L.seg_end.assign(L.segs.size(), 0);
          if (cudaMemsetAsync(S->d_counter + sidx, 0, sizeof(unsigned long long), strm) != cudaSuccess ||
              cudaMemcpyAsync(S->d_stop + sidx, S->h_flags, sizeof(unsigned int), cudaMemcpyHostToDevice,
                              strm) != cudaSuccess) {
            rc = chem::cuda_fail(cudaGetLastError(), "server counter / stop flag");
          } else {
            rc = chem::launch_advance_slice(L.mech, L.segs.data(), (int)L.segs.size(), S->slice_ns,
                                            S->d_counter + sidx, L.seg_end.data(), strm, S->d_stop + sidx,
                                            kMinSliceNs);
            L.issued_total = L.seg_end.back();
          }
          if (rc == CHEM_OK &&
              cudaMemcpyAsync(S->h_counter + sidx, S->d_counter + sidx, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, strm) != cudaSuccess)
            rc = chem::cuda_fail(cudaGetLastError(), "cudaMemcpyAsync(server counter)");
        } else {
          std::vector<chem_segment> segs;
          for (uint64_t id : grp) {
            const Req& r = S->reqs[id];
            const StateRec& st = S->states[r.state];
            chem_segment g{};
            g.T = st.T; g.p = st.p; g.Y = st.Y; g.ld = st.ld; g.ncells = st.ncells;
            g.dt = r.dt; g.rtol = r.rtol; g.atol = r.atol;
            segs.push_back(g);
          }
          const StateRec& st0 = S->states[r0.state];
          // running FP64 slices stop claiming cells (after their minimum time), so that this
          // pass's kernels get the SMs as the slices' cells in flight finish; the copies run on
          // this pass's stream, ahead of its kernels
          for (const Launch& F : S->launches)
            if (F.sliced && cudaEventQuery(F.ev) == cudaErrorNotReady &&
                cudaMemcpyAsync(S->d_stop + F.stream, S->h_flags + 1, sizeof(unsigned int), cudaMemcpyHostToDevice,
                                strm) != cudaSuccess)
              rc = chem::cuda_fail(cudaGetLastError(), "cudaMemcpyAsync(server stop flag)");
          if (rc == CHEM_OK)
            rc = chem_surrogate_advance_batch(st0.model, st0.mech, segs.data(), (int)segs.size(), strm);
        }
        const Clock::time_point now = Clock::now();
        if (rc != CHEM_OK) {
          const char* msg = chem_last_error();
          for (uint64_t id : grp) {
            Req& r = S->reqs[id];
            r.status = Q_FAILED;
            r.error = msg ? msg : "launch failed";
            r.t_done = now;
            S->states[r.state].busy = false;
            ++S->n_failed;
          }
          S->cv_done.notify_all();
          launched = true;
          continue;
        }
        L.stream = sidx;
        L.reqs = grp;
        L.bytes = bytes;
        cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
        cudaEventRecord(L.ev, strm);
        for (uint64_t id : grp) S->reqs[id].status = Q_RUNNING;
        S->inflight += bytes;
        S->stream_busy[sidx] = true;
        S->launches.push_back(L);
        ++S->n_launches;
        if (L.sliced) ++S->n_slices;
        S->n_batched += (int64_t)grp.size();
        S->max_concurrent = std::max<int64_t>(S->max_concurrent, (int64_t)S->launches.size());
        launched = true;
      }
      for (auto it = back.rbegin(); it != back.rend(); ++it) S->pending.push_front(*it);
      // groups that found no free stream wait (below) for a launch to retire, with the lock released
      if (launched) continue;
    }
    // ---- wait ----
    if (S->launches.empty()) {
      // nothing runs, so every queued request that fits was just launched: what is left can never
      // fit (states registered after it took the budget) and fails rather than waiting forever
      if (!S->stop && !S->pending.empty()) {
        const Clock::time_point now = Clock::now();
        for (uint64_t id : S->pending) {
          Req& r = S->reqs[id];
          r.status = Q_FAILED;
          r.error = "request no longer fits the memory budget left by the resident states";
          r.t_done = now;
          ++S->n_failed;
        }
        S->pending.clear();
        S->cv_done.notify_all();
      }
      S->cv_work.wait(lk, [&] { return S->stop || S->n_submitted != submitted; });
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds((int)S->idle_poll_us));
      lk.lock();
    }
  }
}

}  // namespace

using namespace chem;

extern "C" int chem_serve_create(size_t hbm_budget_bytes, const chem_serve_options* opt, chem_server_t* out) {
  if (!out || hbm_budget_bytes == 0) { set_error("bad arguments"); return CHEM_EINVAL; }
  *out = nullptr;
  chem_server_s* S = new chem_server_s();
  S->budget = hbm_budget_bytes;
  const int nfp = (opt && opt->n_streams > 0) ? opt->n_streams : 4;
  const int ns = 2 * nfp;          // nfp low-priority FP64 streams + nfp high-priority surrogate streams
  S->n_fp64 = nfp;
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (opt && opt->idle_poll_us > 0) S->idle_poll_us = opt->idle_poll_us;
  if (opt && opt->slice_ms != 0.0)
    S->slice_ns = opt->slice_ms < 0.0 ? 0ull : (unsigned long long)(opt->slice_ms * 1e6);
  if (opt && opt->max_pause_ms != 0.0)
    S->max_pause_ns = opt->max_pause_ms < 0.0 ? 0ull : (unsigned long long)(opt->max_pause_ms * 1e6);
  if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return cuda_fail(cudaGetLastError(), "cudaGetDevice"); }
  // device: the counters, then the stop words; pinned host: counter copies, reset values, {0, 1}.
  // Both device words of a stream are set on that stream before each slice it runs (nothing here
  // writes them: a synchronous memset would run on the legacy default stream, unordered with the
  // server's non-blocking streams, and could land in the middle of a job)
  cudaError_t ea = cudaMalloc((void**)&S->d_counter, ns * (sizeof(unsigned long long) + sizeof(unsigned int)));
  cudaError_t eh = ea == cudaSuccess ? cudaHostAlloc((void**)&S->h_counter, (2 * ns + 1) * sizeof(unsigned long long),
                                                     cudaHostAllocDefault)
                                     : ea;
  if (ea != cudaSuccess || eh != cudaSuccess) {
    if (S->d_counter) cudaFree(S->d_counter);
    delete S;
    return cuda_fail(ea != cudaSuccess ? ea : eh, "server counters");
  }
  S->h_reset = S->h_counter + ns;
  S->d_stop = (unsigned int*)(S->d_counter + ns);
  S->h_flags = (unsigned int*)(S->h_counter + 2 * ns);
  S->h_flags[0] = 0u;
  S->h_flags[1] = 1u;
  for (int i = 0; i < ns; ++i) {
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, i < nfp ? prio_low : prio_high);
    if (e != cudaSuccess) {
      for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
      cudaFree(S->d_counter);
      cudaFreeHost(S->h_counter);
      delete S;
      return cuda_fail(e, "cudaStreamCreate");
    }
    S->streams.push_back(st);
    S->stream_busy.push_back(false);
  }
  S->th = std::thread(server_loop, S);
  *out = S;
  return CHEM_OK;
}

extern "C" int chem_serve_register_state(chem_server_t S, chem_mech_t m, chem_model_t model, double* T, double* p,
                                         double* Y, int64_t ld, int64_t ncells, int* state_id) {
  if (!S || !m || !T || !p || !Y || !state_id || ncells <= 0 || ld < ncells) {
    set_error("bad arguments");
    return CHEM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  StateRec st;
  st.mech = m; st.model = model; st.T = T; st.p = p; st.Y = Y; st.ld = ld; st.ncells = ncells;
  st.resident = (size_t)ncells * (m->ns + 2) * sizeof(double);
  if (S->resident + st.resident > S->budget) {
    set_error("state of %zu bytes does not fit the budget", st.resident);
    return CHEM_EBUSY;
  }
  S->resident += st.resident;
  const int id = S->next_state++;
  S->states[id] = st;
  *state_id = id;
  return CHEM_OK;
}

extern "C" int chem_serve_submit(chem_server_t S, int state_id, int route, double dt, double rtol, double atol,
                                 uint64_t* req_id) {
  if (!S || !req_id || !(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) ||
      (route != CHEM_ROUTE_FP64 && route != CHEM_ROUTE_SURROGATE)) {
    set_error("bad arguments");
    return CHEM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->states.find(state_id);
  if (it == S->states.end()) { set_error("unknown state %d", state_id); return CHEM_ENOTFOUND; }
  if (route == CHEM_ROUTE_SURROGATE && !it->second.model) {
    set_error("state %d has no surrogate model", state_id);
    return CHEM_EINVAL;
  }
  Req r;
  r.id = S->next_req++;
  r.state = state_id; r.route = route; r.dt = dt; r.rtol = rtol; r.atol = atol;
  r.bytes = request_bytes(it->second, route);
  if (r.bytes > S->budget - S->resident) {
    set_error("request needs %zu bytes beyond the resident states; budget left %zu", r.bytes,
              S->budget - S->resident);
    return CHEM_EBUSY;
  }
  r.t_submit = Clock::now();
  S->reqs[r.id] = r;
  S->pending.push_back(r.id);
  ++S->n_submitted;
  *req_id = r.id;
  S->cv_work.notify_one();
  return CHEM_OK;
}

extern "C" int chem_serve_poll(chem_server_t S, uint64_t req_id, int* state, double* latency_s) {
  if (!S || !state) { set_error("bad arguments"); return CHEM_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(req_id);
  if (it == S->reqs.end()) { set_error("unknown request"); return CHEM_ENOTFOUND; }
  *state = it->second.status;
  if (latency_s)
    *latency_s = it->second.status >= Q_DONE
                     ? std::chrono::duration<double>(it->second.t_done - it->second.t_submit).count()
                     : -1.0;
  if (it->second.status == Q_FAILED) set_error("%s", it->second.error.c_str());
  return CHEM_OK;
}

extern "C" int chem_serve_wait(chem_server_t S, uint64_t req_id, double timeout_s) {
  if (!S || timeout_s < 0) { set_error("bad arguments"); return CHEM_EINVAL; }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(req_id);
  if (it == S->reqs.end()) { set_error("unknown request"); return CHEM_ENOTFOUND; }
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  const bool ok = S->cv_done.wait_until(lk, deadline, [&] { return S->reqs[req_id].status >= Q_DONE; });
  if (!ok) { set_error("request %llu not finished within %g s", (unsigned long long)req_id, timeout_s); return CHEM_ETIMEOUT; }
  if (S->reqs[req_id].status == Q_FAILED) { set_error("%s", S->reqs[req_id].error.c_str()); return CHEM_ECUDA; }
  return CHEM_OK;
}

extern "C" int chem_serve_stats(chem_server_t S, int64_t* out /*[8]*/) {
  if (!S || !out) { set_error("bad arguments"); return CHEM_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->n_done; out[1] = S->n_failed; out[2] = S->n_launches; out[3] = S->n_batched;
  out[4] = S->max_concurrent; out[5] = (int64_t)(S->resident + S->inflight);
  out[6] = S->n_slices; out[7] = S->n_joined;
  return CHEM_OK;
}

extern "C" int chem_serve_destroy(chem_server_t S) {
  if (!S) { set_error("NULL server"); return CHEM_EINVAL; }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    // queued requests that never started are dropped as failed
    const Clock::time_point now = Clock::now();
    for (uint64_t id : S->pending) {
      Req& r = S->reqs[id];
      r.status = Q_FAILED;
      r.error = "server destroyed";
      r.t_done = now;
      ++S->n_failed;
    }
    S->pending.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  if (S->th.joinable()) S->th.join();
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  cudaFree(S->d_counter);
  cudaFreeHost(S->h_counter);
  delete S;
  return CHEM_OK;
}
