// Batched frames of uneven requests: many requests of mixed image size, J, D/r0
// and P2S form, each with several frames of independent Philox streams (the
// serving pattern of the frame pipeline of Fig. dfp2s).
//
// The engine keeps, per shape class (J, C, H, W), a frame context (its scratch
// sized to the class) on a spectral factor shared by every class of the same
// (J, N); the factor and the context are built the first time the class
// appears, and so is the class's choice of field column-pass kernel (the
// autotuner: each candidate timed on the class's own frames with CUDA events,
// the faster kept and reported).  A run enqueues the frames of each class in
// turn on the engine's own stream; with graphs on, the frames of a class are
// captured into one CUDA graph (tens to thousands of kernel launches) that is
// updated in place when the next run has the same shape of work, and launched
// once.  The big kernels of a frame are persistent already (one CTA per SM
// looping over tiles).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace {

struct EngineClass {
  int J = 0, C = 0, H = 0, W = 0, N = 0;
  const dfp2s_p2s* p = nullptr;
  dfp2s_ctx* ctx = nullptr;
  int variant = -1;                   // field column-pass kernel in use
  float tuned_ms[2] = {-1.f, -1.f};   // ms per frame of each candidate (-1: not timed)
  bool warm[3] = {false, false, false};  // a frame of this P2S form has run outside a capture
  cudaGraphExec_t exec = nullptr;     // the class's frames of the last run
  int exec_frames = 0;
};

}  // namespace

struct dfp2s_engine {
  std::vector<const dfp2s_p2s*> p2s;
  double ppd = 8.0;
  int flags = 0;
  cudaStream_t work = nullptr;
  cudaEvent_t in_ev = nullptr, out_ev = nullptr;
  std::map<std::pair<int, int>, dfp2s_factor*> factors;  // (J, N)
  std::vector<EngineClass> classes;
  long long frames_run = 0, graph_launches = 0, graph_updates = 0, graph_instantiations = 0;
};

namespace {

void engine_free(dfp2s_engine* e) {
  if (!e) return;
  for (EngineClass& k : e->classes) {
    if (k.exec) cudaGraphExecDestroy(k.exec);
    dfp2s_ctx_destroy(k.ctx);
  }
  for (auto& f : e->factors) dfp2s_factor_destroy(f.second);
  if (e->in_ev) cudaEventDestroy(e->in_ev);
  if (e->out_ev) cudaEventDestroy(e->out_ev);
  if (e->work) cudaStreamDestroy(e->work);
  delete e;
}

const dfp2s_p2s* p2s_for(const dfp2s_engine* e, int J) {
  for (const dfp2s_p2s* p : e->p2s)
    if (p->d.J == J) return p;
  return nullptr;
}

// The class of a request, created (factor, context) on first use; -1 on failure (message set).
int class_of(dfp2s_engine* e, const dfp2s_request& r) {
  for (size_t i = 0; i < e->classes.size(); ++i) {
    const EngineClass& k = e->classes[i];
    if (k.J == r.J && k.C == r.C && k.H == r.H && k.W == r.W) return (int)i;
  }
  EngineClass k;
  k.J = r.J;
  k.C = r.C;
  k.H = r.H;
  k.W = r.W;
  k.p = p2s_for(e, r.J);
  k.N = dfp2s_grid_size(r.H, r.W, e->ppd);
  if (k.N < 0) return -1;
  dfp2s_factor*& f = e->factors[std::make_pair(k.J, k.N)];
  if (!f) {
    dfp2s_factor_params fp = {k.J, k.N, e->ppd, DFP2S_FACTOR_FACTORED};
    if (dfp2s_build_spectral_factor(&fp, &f, e->work) != DFP2S_OK) {
      e->factors.erase(std::make_pair(k.J, k.N));
      return -1;
    }
  }
  if (dfp2s_ctx_create(f, k.p, k.C, k.H, k.W, &k.ctx) != DFP2S_OK) return -1;
  e->classes.push_back(k);
  return (int)e->classes.size() - 1;
}

// Runs one frame of each P2S form the class has not run yet, outside any capture (first-use allocations and
// weight packing happen here), then, with autotuning on and on first use, times each column-pass candidate on
// three frames of the class and keeps the faster.
int warm_and_tune(dfp2s_engine* e, EngineClass& k, const dfp2s_request& r) {
  if (!k.warm[r.p2s_mode]) {
    const int rc = dfp2s_simulate_frame(k.ctx, r.img_dev, r.C, r.H, r.W, r.D_over_r0, r.seed, r.first_frame,
                                        r.p2s_mode, r.out_dev, e->work);
    if (rc != DFP2S_OK) return rc;
    k.warm[r.p2s_mode] = true;
  }
  if (!(e->flags & DFP2S_ENGINE_AUTOTUNE) || k.tuned_ms[0] >= 0.f) return DFP2S_OK;
  const int ncand = k.N <= 2048 ? 2 : 1;
  cudaEvent_t t0, t1;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    return dfp2s_fail(DFP2S_ECUDA, "autotuner events");
  int rc = DFP2S_OK;
  for (int v = 0; v < ncand && rc == DFP2S_OK; ++v) {
    dfp2s_ctx_set_field_variant(k.ctx, v);
    for (int i = 0; i < 4 && rc == DFP2S_OK; ++i) {  // one untimed frame, then three timed
      if (i == 1) cudaEventRecord(t0, e->work);
      rc = dfp2s_simulate_frame(k.ctx, r.img_dev, r.C, r.H, r.W, r.D_over_r0, r.seed, r.first_frame, r.p2s_mode,
                                r.out_dev, e->work);
    }
    cudaEventRecord(t1, e->work);
    float ms = 0.f;
    if (rc == DFP2S_OK && cudaEventSynchronize(t1) == cudaSuccess && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess)
      k.tuned_ms[v] = ms / 3.f;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc != DFP2S_OK) return rc;
  k.variant = (ncand == 2 && k.tuned_ms[1] >= 0.f && k.tuned_ms[1] < k.tuned_ms[0]) ? 1 : 0;
  dfp2s_ctx_set_field_variant(k.ctx, k.variant);
  return DFP2S_OK;
}

}  // namespace

extern "C" int dfp2s_engine_create(const dfp2s_p2s* const* p2s, int n_p2s, double pix_per_D, int flags,
                                   dfp2s_engine** out) {
  if (!out || !p2s || n_p2s < 1 || n_p2s > 16) return dfp2s_fail(DFP2S_EINVAL, "bad P2S handle list");
  *out = nullptr;
  if (!(pix_per_D > 0 && pix_per_D <= 64)) return dfp2s_fail(DFP2S_EINVAL, "pix_per_D out of range");
  if (flags & ~(DFP2S_ENGINE_GRAPHS | DFP2S_ENGINE_AUTOTUNE)) return dfp2s_fail(DFP2S_EINVAL, "unknown flags");
  dfp2s_engine* e = new dfp2s_engine();
  for (int i = 0; i < n_p2s; ++i) {
    if (!p2s[i] || p2s_for(e, p2s[i]->d.J)) {
      delete e;
      return dfp2s_fail(DFP2S_EINVAL, "P2S handle %d is null or repeats a J", i);
    }
    e->p2s.push_back(p2s[i]);
  }
  e->ppd = pix_per_D;
  e->flags = flags;
  cudaError_t err;
  if ((err = cudaStreamCreateWithFlags(&e->work, cudaStreamNonBlocking)) != cudaSuccess ||
      (err = cudaEventCreateWithFlags(&e->in_ev, cudaEventDisableTiming)) != cudaSuccess ||
      (err = cudaEventCreateWithFlags(&e->out_ev, cudaEventDisableTiming)) != cudaSuccess) {
    engine_free(e);
    return dfp2s_fail_cuda(err, "engine stream");
  }
  *out = e;
  return DFP2S_OK;
}

extern "C" int dfp2s_engine_destroy(dfp2s_engine* e) {
  if (e) cudaStreamSynchronize(e->work);
  engine_free(e);
  return DFP2S_OK;
}

extern "C" int dfp2s_engine_run(dfp2s_engine* e, const dfp2s_request* req, int n_req, void* stream) {
  if (!e || (!req && n_req > 0) || n_req < 0) return dfp2s_fail(DFP2S_EINVAL, "null argument");
  for (int i = 0; i < n_req; ++i) {
    const dfp2s_request& r = req[i];
    if (!r.img_dev || !r.out_dev || r.n_frames < 0 || r.C < 1 || r.C > 64 || r.H < 1 || r.W < 1 || r.H > 4096 ||
        r.W > 4096)
      return dfp2s_fail(DFP2S_EINVAL, "request %d: bad buffers or shape", i);
    if (!(r.D_over_r0 >= 0 && r.D_over_r0 <= 1e4)) return dfp2s_fail(DFP2S_EINVAL, "request %d: bad D/r0", i);
    if (r.p2s_mode != DFP2S_P2S_EXACT && r.p2s_mode != DFP2S_P2S_LEARNED && r.p2s_mode != DFP2S_P2S_LEARNED_FP32)
      return dfp2s_fail(DFP2S_EINVAL, "request %d: unknown P2S mode", i);
    const dfp2s_p2s* p = p2s_for(e, r.J);
    if (!p) return dfp2s_fail(DFP2S_EINVAL, "request %d: no P2S handle for J = %d", i, r.J);
    if (r.p2s_mode != DFP2S_P2S_EXACT && !p->d.has_mlp)
      return dfp2s_fail(DFP2S_EINVAL, "request %d: no surrogate network for J = %d", i, r.J);
  }
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  // the engine's stream follows the caller's, and the caller's follows the engine's at the end
  if (cudaEventRecord(e->in_ev, user) != cudaSuccess || cudaStreamWaitEvent(e->work, e->in_ev, 0) != cudaSuccess)
    return dfp2s_fail_cuda(cudaGetLastError(), "engine stream order");
  // classes (created on first use), the requests of each, largest frames first (so that the P2S handles' shared
  // blur scratch is sized once)
  std::vector<int> cls(n_req);
  for (int i = 0; i < n_req; ++i)
    if ((cls[i] = class_of(e, req[i])) < 0) return dfp2s_last_error(nullptr, 0);  // the failure's own code
  std::vector<int> order;
  for (int i = 0; i < (int)e->classes.size(); ++i)
    if (std::find(cls.begin(), cls.end(), i) != cls.end()) order.push_back(i);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const EngineClass &ka = e->classes[a], &kb = e->classes[b];
    return (long long)ka.C * ka.H * ka.W > (long long)kb.C * kb.H * kb.W;
  });
  for (int ci : order)
    for (int i = 0; i < n_req; ++i)
      if (cls[i] == ci && req[i].n_frames > 0) {
        const int rc = warm_and_tune(e, e->classes[ci], req[i]);
        if (rc != DFP2S_OK) return rc;
      }
  for (int ci : order) {
    EngineClass& k = e->classes[ci];
    int nfr = 0;
    for (int i = 0; i < n_req; ++i)
      if (cls[i] == ci) nfr += req[i].n_frames;
    if (nfr == 0) continue;
    const bool graphs = (e->flags & DFP2S_ENGINE_GRAPHS) != 0;
    if (graphs && cudaStreamBeginCapture(e->work, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return dfp2s_fail_cuda(cudaGetLastError(), "engine graph capture");
    int rc = DFP2S_OK;
    for (int i = 0; i < n_req && rc == DFP2S_OK; ++i) {
      if (cls[i] != ci) continue;
      const dfp2s_request& r = req[i];
      const size_t frame_elems = (size_t)r.C * r.H * r.W;
      for (int f = 0; f < r.n_frames && rc == DFP2S_OK; ++f)
        rc = dfp2s_simulate_frame(k.ctx, r.img_dev, r.C, r.H, r.W, r.D_over_r0, r.seed, r.first_frame + (uint32_t)f,
                                  r.p2s_mode, r.out_dev + (size_t)f * frame_elems, e->work);
    }
    if (graphs) {
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(e->work, &g);
      if (rc != DFP2S_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) return dfp2s_fail_cuda(ce, "engine graph capture");
      bool updated = false;
      if (k.exec && k.exec_frames == nfr) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(k.exec, g, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();  // clear the failed update's error
      }
      if (!updated) {
        if (k.exec) cudaGraphExecDestroy(k.exec);
        k.exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&k.exec, g, 0);
        if (ie != cudaSuccess) {
          cudaGraphDestroy(g);
          return dfp2s_fail_cuda(ie, "engine graph instantiation");
        }
        k.exec_frames = nfr;
        ++e->graph_instantiations;
      } else {
        ++e->graph_updates;
      }
      cudaGraphDestroy(g);
      const cudaError_t le = cudaGraphLaunch(k.exec, e->work);
      if (le != cudaSuccess) return dfp2s_fail_cuda(le, "engine graph launch");
      ++e->graph_launches;
    } else if (rc != DFP2S_OK) {
      return rc;
    }
    e->frames_run += nfr;
  }
  if (cudaEventRecord(e->out_ev, e->work) != cudaSuccess || cudaStreamWaitEvent(user, e->out_ev, 0) != cudaSuccess)
    return dfp2s_fail_cuda(cudaGetLastError(), "engine stream order");
  return DFP2S_OK;
}

extern "C" int dfp2s_engine_info(const dfp2s_engine* e, int* n_classes, long long* counters_host) {
  if (!e) return dfp2s_fail(DFP2S_EINVAL, "null engine");
  if (n_classes) *n_classes = (int)e->classes.size();
  if (counters_host) {
    counters_host[0] = e->frames_run;
    counters_host[1] = e->graph_launches;
    counters_host[2] = e->graph_instantiations;
    counters_host[3] = e->graph_updates;
  }
  return DFP2S_OK;
}

extern "C" int dfp2s_engine_class_info(const dfp2s_engine* e, int i, int* shape_host, float* tuned_ms_host) {
  if (!e || i < 0 || i >= (int)e->classes.size()) return dfp2s_fail(DFP2S_EINVAL, "no class %d", i);
  const EngineClass& k = e->classes[i];
  if (shape_host) {
    const int v[6] = {k.J, k.C, k.H, k.W, k.N, k.variant};
    memcpy(shape_host, v, sizeof(v));
  }
  if (tuned_ms_host) {
    tuned_ms_host[0] = k.tuned_ms[0];
    tuned_ms_host[1] = k.tuned_ms[1];
  }
  return DFP2S_OK;
}
