// Context, status strings and error recording of the C ABI.

#include "common.cuh"

#include <new>
#include <string.h>

int tb_fail(tb_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->last_error, sizeof(ctx->last_error), fmt, ap);
    va_end(ap);
  }
  return code;
}

extern "C" const char* tb_status_string(int status) {
  switch (status) {
    case TB_OK: return "ok";
    case TB_ERR_ARG: return "invalid argument";
    case TB_ERR_NOT_CONVERGED: return "not converged";
    case TB_ERR_GAP: return "no gap at the occupation";
    case TB_ERR_OOM: return "capacity exceeded";
    case TB_ERR_TIMEOUT: return "device wait timed out";
    case TB_ERR_CUDA: return "CUDA error";
    case TB_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

extern "C" const char* tb_ctx_last_error(const tb_ctx* ctx) { return ctx ? ctx->last_error : "null context"; }

extern "C" int tb_ctx_create(tb_ctx** out) {
  if (!out) return TB_ERR_ARG;
  *out = nullptr;
  tb_ctx* ctx = new (std::nothrow) tb_ctx();
  if (!ctx) return TB_ERR_OOM;
  ctx->last_error[0] = 0;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return TB_ERR_CUDA;
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return TB_ERR_CUDA;
  }
  ctx->sm_count = prop.multiProcessorCount;
  ctx->grid_limit = 0;
  ctx->sp2_form = TB_SP2_FORM_AUTO;
  ctx->pair_clusters = -1;
  ctx->oz_pair_clusters = -1;
  ctx->wait_ns = 2000000000ull;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;
  if (!(prop.major == 10 && prop.minor == 3)) {
    delete ctx;
    return TB_ERR_UNSUPPORTED;
  }
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  ctx->encode_tiled = (e == cudaSuccess && q == cudaDriverEntryPointSuccess)
                          ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                          : nullptr;
  *out = ctx;
  return TB_OK;
}

int tb_loop_begin(tb_ctx* ctx, cudaStream_t s, DevLoop* L) {
  *L = DevLoop{};
  L->outer = s;
  L->body_stream = s;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  TB_CUDA_TRY(ctx, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return TB_OK;
  if (!ctx->loop_stream) TB_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->loop_stream, cudaStreamNonBlocking));
  TB_CUDA_TRY(ctx, cudaGraphConditionalHandleCreate(&L->handle, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = L->handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  TB_CUDA_TRY(ctx, cudaGraphAddNode(&L->node, g, deps, nullptr, nd, &np));
  TB_CUDA_TRY(ctx, cudaStreamUpdateCaptureDependencies(s, &L->node, nullptr, 1, cudaStreamSetCaptureDependencies));
  TB_CUDA_TRY(ctx, cudaStreamBeginCaptureToGraph(ctx->loop_stream, np.conditional.phGraph_out[0], nullptr, nullptr,
                                                 0, cudaStreamCaptureModeRelaxed));
  L->graph = 1;
  L->body_stream = ctx->loop_stream;
  return TB_OK;
}

int tb_loop_end(tb_ctx* ctx, DevLoop* L, int rc) {
  if (!L->graph) return rc;
  L->graph = 0;
  cudaGraph_t body = nullptr;
  const cudaError_t e = cudaStreamEndCapture(L->body_stream, &body);
  if (rc) return rc;
  if (e != cudaSuccess) return tb_fail(ctx, TB_ERR_CUDA, "loop body capture: %s", cudaGetErrorString(e));
  return TB_OK;
}

extern "C" int tb_ctx_destroy(tb_ctx* ctx) {
  if (ctx && ctx->loop_stream) cudaStreamDestroy(ctx->loop_stream);
  if (ctx && ctx->prof_created) {
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i <= TB_PROF_MAX; ++i) cudaEventDestroy(ctx->ev[p][i]);
  }
  delete ctx;
  return TB_OK;
}

extern "C" int tb_ctx_set_profiling(tb_ctx* ctx, int enable) {
  if (!ctx) return TB_ERR_ARG;
  if (enable && !ctx->prof_created) {
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i <= TB_PROF_MAX; ++i) TB_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev[p][i]));
    ctx->prof_created = 1;
  }
  if (enable) ctx->prof_on = 1;
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  if (!enable) ctx->prof_on = 0;
  return TB_OK;
}

extern "C" int tb_ctx_set_grid_limit(tb_ctx* ctx, int max_ctas) {
  if (!ctx) return TB_ERR_ARG;
  if (max_ctas < 0) return tb_fail(ctx, TB_ERR_ARG, "grid limit %d < 0", max_ctas);
  ctx->grid_limit = max_ctas;
  return TB_OK;
}

extern "C" int tb_ctx_set_sp2_form(tb_ctx* ctx, int form) {
  if (!ctx) return TB_ERR_ARG;
  if (form < TB_SP2_FORM_AUTO || form > TB_SP2_FORM_PAIRS) return tb_fail(ctx, TB_ERR_ARG, "sp2 form %d", form);
  ctx->sp2_form = form;
  return TB_OK;
}

extern "C" int tb_ctx_set_wait_limit(tb_ctx* ctx, unsigned long long ns) {
  if (!ctx) return TB_ERR_ARG;
  if (ns < 1 || ns > 2000000000ull) return tb_fail(ctx, TB_ERR_ARG, "wait limit %llu ns outside 1..2e9", ns);
  ctx->wait_ns = ns;
  return TB_OK;
}

extern "C" int tb_ctx_sp2_launch_times(tb_ctx* ctx, int phase, float* ms, int cap, int* count) {
  if (!ctx || phase < 0 || phase > 1 || !count) return TB_ERR_ARG;
  *count = 0;
  if (!ctx->prof_on) return TB_OK;
  const int n = ctx->prof_n[phase] - 1;  // events bracket n launches
  if (n <= 0) return TB_OK;
  TB_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev[phase][n]));
  const int m = n < cap ? n : cap;
  for (int i = 0; i < m; ++i) TB_CUDA_TRY(ctx, cudaEventElapsedTime(&ms[i], ctx->ev[phase][i], ctx->ev[phase][i + 1]));
  *count = m;
  return TB_OK;
}
