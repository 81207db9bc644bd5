// One "chemistry + thermo" step of the reactive-flow time loop (the paper's Fig. 1 iteration,
// §3.1, restricted to the per-cell stages: chemical source, Thermo, transport properties), issued
// as one stream sequence and, on request, captured once into a CUDA graph and replayed (§3.2:
// the paper captures its per-step kernel sequence in CUDA graphs and takes temporaries from the
// stream-ordered allocator).
//
// Stages of a step, all on the caller's stream:
//   0  thermo in:   copy (T, Y) into the step's start buffers; mixture h0 and cp0 (NASA-7)
//   1  chemistry:   FP64 Rodas4 (chem_advance_ex) or the BF16 surrogate with FP64 fallback
//   2  thermo out:  heat-release rate q of the step; T from h(T, Y1) = h0 by Newton (the adiabatic
//                   constant-pressure step conserves h: the Thermo class recovers T from it)
//   3  transport:   mixture-averaged mu, lambda and D_km of the new state
// Per-stage device times (CUDA events between the stages) are measured on direct runs; a graph
// replay is timed as a whole.
#include <cuda_runtime.h>

#include <cstring>

#include "chem_internal.h"
#include "surrogate_model.h"

using chem::cuda_fail;
using chem::set_error;

struct chem_step_s {
  chem_step_desc d{};
  double* T0 = nullptr;           // start state copies [ld], [ns][ld]
  double* Y0 = nullptr;
  cudaStream_t cap = nullptr;     // private stream the graph is captured on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[5] = {};
  bool timed = false;
};

namespace {

// the stage sequence on stream st; with events, the stage boundaries are recorded in ev
int issue(chem_step_s* s, cudaStream_t st, bool events) {
  const chem_step_desc& d = s->d;
  const int ns = d.mech->ns;
  const int64_t ld = d.ld, n = d.ncells;
  if (events) CHEM_CUDA_TRY(cudaEventRecord(s->ev[0], st));
  CHEM_CUDA_TRY(cudaMemcpyAsync(s->T0, d.T, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
  CHEM_CUDA_TRY(cudaMemcpy2DAsync(s->Y0, (size_t)ld * 8, d.Y, (size_t)ld * 8, (size_t)n * 8, ns,
                                  cudaMemcpyDeviceToDevice, st));
  int rc = chem_mixture_thermo(d.mech, s->T0, s->Y0, ld, n, d.h0, d.cp0, st);
  if (rc) return rc;
  if (events) CHEM_CUDA_TRY(cudaEventRecord(s->ev[1], st));
  if (d.model)
    rc = chem_surrogate_advance(d.model, d.mech, d.T, d.p, d.Y, ld, d.dt, n, d.rtol, d.atol, d.route, st);
  else
    rc = chem_advance_ex(d.mech, d.T, d.p, d.Y, ld, d.dt, n, d.rtol, d.atol, nullptr, d.status, d.nsub,
                         nullptr, nullptr, st);
  if (rc < 0) return rc;
  if (events) CHEM_CUDA_TRY(cudaEventRecord(s->ev[2], st));
  if (d.q) {
    rc = chem_heat_release(d.mech, s->T0, d.p, s->Y0, d.Y, ld, n, d.dt, d.q, st);
    if (rc) return rc;
  }
  rc = chem_temperature_from_enthalpy(d.mech, d.h0, d.Y, ld, n, d.T, d.thermo_status, st);
  if (rc) return rc;
  if (events) CHEM_CUDA_TRY(cudaEventRecord(s->ev[3], st));
  if (d.transport) {
    rc = chem_transport_eval(d.transport, d.T, d.p, d.Y, ld, n, d.mu, d.lambda, d.Dmix, st);
    if (rc) return rc;
  }
  if (events) CHEM_CUDA_TRY(cudaEventRecord(s->ev[4], st));
  return CHEM_OK;
}

}  // namespace

extern "C" int chem_step_free(chem_step_t s) {
  if (!s) { set_error("NULL step"); return CHEM_EINVAL; }
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->cap) cudaStreamDestroy(s->cap);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->T0) cudaFree(s->T0);
  if (s->Y0) cudaFree(s->Y0);
  delete s;
  return CHEM_OK;
}

extern "C" int chem_step_create(const chem_step_desc* d, chem_step_t* out) {
  if (!d || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  *out = nullptr;
  if (!d->mech || d->ncells < 1 || d->ld < d->ncells || !d->T || !d->p || !d->Y || !d->h0 ||
      !(d->dt > 0.0) || !(d->rtol > 0.0) || !(d->atol > 0.0)) {
    set_error("step: a mechanism, ncells >= 1, ld >= ncells, T, p, Y, h0 and positive dt, rtol, atol are "
              "required");
    return CHEM_EINVAL;
  }
  if (d->model && d->model->ns != d->mech->ns) { set_error("step: model and mechanism disagree"); return CHEM_EINVAL; }
  if (d->transport && !d->mu && !d->lambda && !d->Dmix) {
    set_error("step: transport given without an output");
    return CHEM_EINVAL;
  }
  chem_step_s* s = new chem_step_s();
  s->d = *d;
  auto fail = [&](cudaError_t e, const char* what) { chem_step_free(s); return cuda_fail(e, what); };
  cudaError_t e = cudaMalloc((void**)&s->T0, (size_t)d->ncells * 8);
  if (e) return fail(e, "cudaMalloc(step)");
  e = cudaMalloc((void**)&s->Y0, (size_t)d->ld * d->mech->ns * 8);
  if (e) return fail(e, "cudaMalloc(step)");
  for (cudaEvent_t& ev : s->ev)
    if ((e = cudaEventCreate(&ev))) return fail(e, "cudaEventCreate");
  if ((e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking))) return fail(e, "cudaStreamCreate");
  *out = s;
  return CHEM_OK;
}

extern "C" int chem_step_run(chem_step_t s, int use_graph, chem_stream_t stream) {
  if (!s) { set_error("NULL step"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  if (!use_graph) {
    int rc = issue(s, st, true);
    if (rc) return rc;
    s->timed = true;
    return CHEM_OK;
  }
  if (!s->exec) {
    // capture once on the private stream (capturing runs nothing), then instantiate
    CHEM_CUDA_TRY(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    int rc = issue(s, s->cap, false);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(s->cap, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
    s->graph = g;
    CHEM_CUDA_TRY(cudaGraphInstantiate(&s->exec, g, 0));
  }
  CHEM_CUDA_TRY(cudaGraphLaunch(s->exec, st));
  return CHEM_OK;
}

extern "C" int chem_step_stage_ms(chem_step_t s, float* ms) {
  if (!s || !ms) { set_error("NULL argument"); return CHEM_EINVAL; }
  if (!s->timed) { set_error("no direct step has run yet"); return CHEM_EINVAL; }
  CHEM_CUDA_TRY(cudaEventSynchronize(s->ev[4]));
  for (int i = 0; i < 4; ++i) CHEM_CUDA_TRY(cudaEventElapsedTime(&ms[i], s->ev[i], s->ev[i + 1]));
  return CHEM_OK;
}
