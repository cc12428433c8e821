// Batches of pure-SHT plane solves (paper Sec. 3.2) on the mixed-precision
// tensor-core path: grouping of planes into (nside, lmax) classes, the
// buffers of a batch, CUDA-graph capture of the six persistent launches and
// the autotuner that picks their launch shapes.
//
// A batch plan owns every intermediate buffer and reads its inputs and
// outputs through device-side pointer tables, so the captured graph stays
// valid for any maps the caller passes: an execution copies the pointer
// tables (pinned host staging, one asynchronous copy) and launches the graph.
#include <algorithm>
#include <cmath>
#include <map>

#include "legendre_tc.cuh"

namespace clc {

int poisson_sht_tc(clc_ctx* ctx, const double* const* kappa, int P, int nside, int lmax, double* const* psi,
                   const clc_derivs* out);

static int round16(int v) { return (v + 15) / 16 * 16; }

struct TcBatch {
  clc_ctx* ctx = nullptr;
  TcBatchDev dev{};
  TcItems items;
  TcLaunch launch;
  std::vector<std::shared_ptr<TcTable>> tabs;
  std::vector<std::shared_ptr<FftPlan>> plans;
  std::vector<int> slot;           // caller's plane index -> slot in the pointer tables
  int nplanes = 0, mode = 0;
  Buffer work, ptrs;
  size_t work_bytes = 0;
  void* h_ptrs = nullptr;          // pinned staging of the pointer tables
  size_t ptr_bytes = 0;
  cudaEvent_t ptr_ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool use_graph = false, tune = false, tuned = false;
  double stage_ms[6] = {0, 0, 0, 0, 0, 0};
  ~TcBatch() {
    if (ptr_ev) {
      cudaEventSynchronize(ptr_ev);
      cudaEventDestroy(ptr_ev);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (h_ptrs) cudaFreeHost(h_ptrs);
  }
};

// Largest number of planes of one class in a batch: the synthesis holds two
// accumulators of round16(2 nq P) FP32 columns in at most 256 TMEM columns.
int tc_class_limit(int mode) { return mode ? 21 : 64; }

static int tc_batch_build(clc_ctx* ctx, int nplanes, const int* nside, const int* lmax, int mode, TcBatch* B) {
  B->ctx = ctx;
  B->nplanes = nplanes;
  B->mode = mode;
  // classes in order of first appearance; a class holds at most
  // tc_class_limit planes, further planes of the same size open a new one
  const int limit = tc_class_limit(mode);
  std::vector<std::pair<int, int>> key;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < nplanes; ++i) {
    if (!valid_nside(nside[i]) || nside[i] < 64 || nside[i] > 4096 || lmax[i] < 1 || lmax[i] > 4 * nside[i])
      return set_err(ctx, CLC_EINVAL, "mixed-precision SHT batch: need 64 <= nside <= 4096 and 1 <= lmax <= 4 nside");
    const auto k = std::make_pair(nside[i], lmax[i]);
    int c = -1;
    for (int j = 0; j < (int)key.size(); ++j)
      if (key[j] == k && (int)members[j].size() < limit) c = j;
    if (c < 0) {
      if ((int)key.size() == kTcMaxClasses)
        return set_err(ctx, CLC_EINVAL, "mixed-precision SHT batch: more than " + std::to_string(kTcMaxClasses) +
                                            " plane classes (at most " + std::to_string(limit) +
                                            " planes of one (nside, lmax) per class)");
      key.push_back(k);
      members.emplace_back();
      c = (int)key.size() - 1;
    }
    members[c].push_back(i);
  }
  const int nq = mode ? 3 : 1;
  TcBatchDev& d = B->dev;
  d.ncls = (int)key.size();
  d.mode = mode;
  B->slot.assign(nplanes, 0);
  // sizes of every class buffer
  struct Sz {
    size_t F, V, Ve, A, S, Se, So, G, G01, Co;
  };
  std::vector<std::vector<double>> co01(key.size());
  std::vector<Sz> sz(d.ncls);
  std::vector<std::vector<long long>> soff(d.ncls);
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t total = 0;
  int plane0 = 0;
  long long ring0 = 0, pa0 = 0, ps0 = 0, low0 = 0;
  int rc = CLC_OK;
  for (int c = 0; c < d.ncls; ++c) {
    const int ns = key[c].first, L = key[c].second, P = (int)members[c].size();
    auto T = get_tc_table(ctx, ns, L, &rc);
    if (rc) return rc;
    auto pl = get_fft_plan(ctx, ns, &rc);
    if (rc) return rc;
    B->tabs.push_back(T);
    B->plans.push_back(pl);
    TcClass& C = d.cls[c];
    C.th = (const __half*)T->hi.p;
    C.tl = (const __half*)T->lo.p;
    C.off = (const long long*)T->off.p;
    C.rows = (const int*)T->rows.p;
    C.pad = (const int*)T->pad.p;
    C.nside = ns;
    C.lmax = L;
    C.R = 2 * ns;
    C.P = P;
    C.nq = nq;
    C.Na = round16(2 * P);
    C.Ns = round16(2 * nq * P);
    C.plane0 = plane0;
    C.wq = 4.0 * kPi / (12.0 * (double)ns * ns);
    C.fft = plan_dev<float>(*pl);
    C.mmax = pl->mmax_fft;
    C.ldf = 4 * ns - 1;
    C.fstride = (size_t)C.ldf * (L + 1);
    C.astride = (size_t)(L + 1) * (L + 2) / 2;
    C.ldm = (L + 1 + 3) / 4 * 4;
    C.qstride = (size_t)C.ldf * C.ldm;
    C.gstride = (size_t)nq * C.qstride;
    C.ring0 = ring0;
    C.pa0 = pa0;
    C.ps0 = ps0;
    C.low0 = low0;
    // recurrence (a_lm, b_lm), eps_lm and -1/(l(l+1)) of the orders m = 0, 1,
    // l = 0 .. lmax + 2; FP64 low orders on the rings with sin(theta) < 0.29
    C.ncap = std::max(1, std::min(2 * ns - 1, (int)std::ceil(0.35 * ns)));
    co01[c].assign(2 * (size_t)(L + 3) * 4, 0.0);
    for (int m = 0; m <= 1; ++m)
      for (int l = 0; l <= L + 2; ++l) {
        double* e = &co01[c][((size_t)m * (L + 3) + l) * 4];
        if (l >= 1) e[3] = -1.0 / ((double)l * (l + 1.0));
        if (l >= m + 2) {
          e[0] = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
          e[1] = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
        }
        if (l > m) e[2] = std::sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0));
      }
    const int G = 2 * (L + 1);
    long long sacc = 0;
    soff[c].resize(G);
    for (int g = 0; g < G; ++g) {
      soff[c][g] = sacc;
      sacc += (long long)C.Ns * T->h_pad[g];
    }
    Sz& z = sz[c];
    z.F = r256(sizeof(float2) * C.fstride * P);
    z.V = r256(sizeof(__half) * (size_t)G * C.R * C.Na);
    z.Ve = r256(sizeof(int) * (size_t)G * C.Na);
    z.A = r256(sizeof(float2) * C.astride * P);
    z.S = r256(sizeof(__half) * (size_t)sacc);
    z.Se = r256(sizeof(int) * (size_t)G * C.Ns);
    z.So = r256(sizeof(long long) * G);
    z.G = r256(sizeof(float2) * C.gstride * P);
    z.G01 = r256(sizeof(double2) * (size_t)P * nq * 2 * C.ldf);
    z.Co = r256(sizeof(double) * co01[c].size());
    total += z.F + 2 * z.V + z.Ve + z.A + 2 * z.S + z.Se + z.So + z.G + z.G01 + z.Co;
    for (int j = 0; j < P; ++j) B->slot[members[c][j]] = plane0 + j;
    plane0 += P;
    ring0 += (long long)P * (4 * ns - 1);
    pa0 += L + 1;
    ps0 += G;
    low0 += (long long)P * C.ncap;
  }
  d.n_ring = ring0;
  d.n_pa = pa0;
  d.n_ps = ps0;
  d.n_low = low0;
  size_t fb = 0, tb = 0;
  cudaMemGetInfo(&fb, &tb);
  if (total + (1ull << 30) > fb)
    return set_err(ctx, CLC_ENOMEM, "mixed-precision SHT batch buffers of " + std::to_string(total >> 20) +
                                        " MiB do not fit");
  B->work.bytes = total;
  if (cudaMalloc(&B->work.p, total) != cudaSuccess) {
    cudaGetLastError();
    B->work.p = nullptr;
    return set_err(ctx, CLC_ENOMEM, "mixed-precision SHT batch allocation failed");
  }
  B->work_bytes = total;
  uint8_t* w = (uint8_t*)B->work.p;
  for (int c = 0; c < d.ncls; ++c) {
    TcClass& C = d.cls[c];
    const Sz& z = sz[c];
    C.F = (float2*)w;
    w += z.F;
    C.vh = (__half*)w;
    w += z.V;
    C.vl = (__half*)w;
    w += z.V;
    C.vexp = (int*)w;
    w += z.Ve;
    C.alm = (float2*)w;
    w += z.A;
    C.sh = (__half*)w;
    w += z.S;
    C.sl = (__half*)w;
    w += z.S;
    C.sexp = (int*)w;
    w += z.Se;
    C.soff = (const long long*)w;
    if ((rc = cuda_check(ctx, cudaMemcpy(w, soff[c].data(), sizeof(long long) * soff[c].size(), cudaMemcpyHostToDevice),
                         "batch layout upload")))
      return rc;
    w += z.So;
    C.G = (float2*)w;
    w += z.G;
    C.G01 = (double2*)w;
    w += z.G01;
    C.co01 = (const double*)w;
    if ((rc = cuda_check(ctx, cudaMemcpy(w, co01[c].data(), sizeof(double) * co01[c].size(), cudaMemcpyHostToDevice),
                         "batch coefficient upload")))
      return rc;
    w += z.Co;
  }
  // pointer tables: kappa[n], out[n][6]
  B->ptr_bytes = sizeof(void*) * (size_t)nplanes * 7;
  B->ptrs.bytes = B->ptr_bytes;
  if (cudaMalloc(&B->ptrs.p, B->ptr_bytes) != cudaSuccess || cudaMallocHost(&B->h_ptrs, B->ptr_bytes) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ptr_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, CLC_ENOMEM, "batch pointer tables");
  }
  d.kappa = (const double* const*)B->ptrs.p;
  d.out = (double* const*)((const double**)B->ptrs.p + nplanes);
  cudaEventRecord(B->ptr_ev, ctx->stream);
  return tc_build_items(ctx, d, B->tabs, &B->items);
}

// Stage the caller's pointers (host arrays of device maps) into the device tables.
static int tc_batch_bind(TcBatch* B, const double* const* kappa, double* const* psi, const clc_derivs* out) {
  clc_ctx* ctx = B->ctx;
  for (int i = 0; i < B->nplanes; ++i)
    if (!kappa[i]) return set_err(ctx, CLC_EINVAL, "SHT batch: NULL kappa map");
  int rc = cuda_check(ctx, cudaEventSynchronize(B->ptr_ev), "pointer staging");
  if (rc) return rc;
  const void** h = (const void**)B->h_ptrs;
  const int n = B->nplanes;
  for (int i = 0; i < n; ++i) {
    const int s = B->slot[i];
    h[s] = kappa[i];
    const void** o = h + n + (size_t)s * 6;
    o[0] = psi ? psi[i] : nullptr;
    for (int f = 1; f < 6; ++f) o[f] = nullptr;
    if (B->mode && out) {
      o[1] = out[i].a_th;
      o[2] = out[i].a_ph;
      o[3] = out[i].u_tt;
      o[4] = out[i].u_pp;
      o[5] = out[i].u_tp;
    }
  }
  rc = cuda_check(ctx, cudaMemcpyAsync(B->ptrs.p, B->h_ptrs, B->ptr_bytes, cudaMemcpyHostToDevice, ctx->stream),
                  "pointer table upload");
  if (rc) return rc;
  return cuda_check(ctx, cudaEventRecord(B->ptr_ev, ctx->stream), "pointer staging event");
}

// Autotuner: each persistent launch is timed (CUDA events, best of two runs
// after a warm-up) for every candidate shape; the fastest is kept.  Stages
// run in pipeline order so each one sees valid inputs, and a tuned stage is
// idempotent (it rewrites the same outputs).
static int tc_autotune(TcBatch* B) {
  clc_ctx* ctx = B->ctx;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = CLC_OK;
  auto time_stage = [&](int stage, const TcLaunch& L, double* ms) -> int {
    int r = tc_run_stage(ctx, B->dev, B->items, L, stage);
    if (r) return r;
    double best = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, ctx->stream);
      r = tc_run_stage(ctx, B->dev, B->items, L, stage);
      if (r) return r;
      cudaEventRecord(e1, ctx->stream);
      if ((r = cuda_check(ctx, cudaEventSynchronize(e1), "autotune timing"))) return r;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, (double)t);
    }
    *ms = best;
    return CLC_OK;
  };
  TcLaunch L = B->launch;
  const int smem_cap = 227 * 1024;
  auto gemm_smem = [](int S, int nmax) { return 1024 + S * (32768 + 2 * ((nmax * 128 + 1023) / 1024 * 1024)); };
  for (int stage = 0; stage < 6 && !rc; ++stage) {
    double best = 1e30;
    TcLaunch pick = L;
    std::vector<TcLaunch> cand;
    if (stage == 0 || stage == 5) {
      for (int c : {2, 4, 8}) {
        TcLaunch x = L;
        x.fft_ctas = c;
        cand.push_back(x);
      }
    } else if (stage == 2 || stage == 4) {
      const int nmax = stage == 2 ? B->items.na_max : B->items.ns_max;
      for (int S = 2; S <= 4; ++S)
        for (int c = 1; c <= 3; ++c) {
          if (gemm_smem(S, nmax) > smem_cap || c * (gemm_smem(S, nmax) + 1024) > 228 * 1024) continue;
          TcLaunch x = L;
          if (stage == 2) {
            x.an_stages = S;
            x.an_ctas = c;
          } else {
            x.sy_stages = S;
            x.sy_ctas = c;
          }
          cand.push_back(x);
        }
    } else {
      cand.push_back(L);
    }
    for (const TcLaunch& x : cand) {
      double ms = 0;
      if ((rc = time_stage(stage, x, &ms))) break;
      if (ms < best) {
        best = ms;
        pick = x;
      }
    }
    if (rc) break;
    L = pick;
    B->stage_ms[stage] = best;
    // leave this stage's outputs from the picked shape for the next stage
    rc = tc_run_stage(ctx, B->dev, B->items, L, stage);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) {
    B->launch = L;
    B->tuned = true;
  }
  return rc;
}

static int tc_batch_execute(TcBatch* B, const double* const* kappa, double* const* psi, const clc_derivs* out) {
  clc_ctx* ctx = B->ctx;
  int rc = tc_batch_bind(B, kappa, psi, out);
  if (rc) return rc;
  if (B->tune && !B->tuned) {
    if ((rc = tc_autotune(B))) return rc;
    if (!B->use_graph) return CLC_OK;   // the tuning pass left every output written
  }
  if (!B->use_graph) return tc_run(ctx, B->dev, B->items, B->launch);
  if (!B->gexec) {
    // capture on a private stream (the context's stream may be the legacy
    // default stream, which cannot be captured); the graph is launched on
    // the context's stream, after the pointer-table upload
    cudaStream_t cs = nullptr;
    if ((rc = cuda_check(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream"))) return rc;
    cudaStream_t user = ctx->stream;
    const bool prof = ctx->prof;
    const long long launches = ctx->launches;
    ctx->prof = false;
    ctx->stream = cs;
    rc = cuda_check(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "graph capture");
    int rrun = CLC_OK;
    cudaError_t ec = cudaSuccess;
    if (!rc) {
      rrun = tc_run(ctx, B->dev, B->items, B->launch);
      ec = cudaStreamEndCapture(cs, &B->graph);
    }
    ctx->stream = user;
    ctx->prof = prof;
    ctx->launches = launches;
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (rrun) return rrun;
    if ((rc = cuda_check(ctx, ec, "graph capture end"))) return rc;
    if ((rc = cuda_check(ctx, cudaGraphInstantiate(&B->gexec, B->graph, 0), "graph instantiate"))) return rc;
  }
  ctx->launches += 6;
  return cuda_check(ctx, cudaGraphLaunch(B->gexec, ctx->stream), "graph launch");
}

// Mixed-precision solve of P planes of one (nside, lmax), through a batch
// layout cached in the context (no graph, default launch shapes).
int poisson_sht_tc(clc_ctx* ctx, const double* const* kappa, int P, int nside, int lmax, double* const* psi,
                   const clc_derivs* out) {
  const int mode = out ? 1 : 0;
  const auto key = std::make_tuple(nside, lmax, P, mode);
  auto it = ctx->tc_batches.find(key);
  std::shared_ptr<TcBatch> B;
  if (it != ctx->tc_batches.end()) {
    B = it->second;
  } else {
    B = std::make_shared<TcBatch>();
    std::vector<int> ns(P, nside), lm(P, lmax);
    const int rc = tc_batch_build(ctx, P, ns.data(), lm.data(), mode, B.get());
    if (rc) return rc;
    ctx->tc_batches[key] = B;
  }
  return tc_batch_execute(B.get(), kappa, psi, out);
}

}  // namespace clc

using namespace clc;

struct clc_sht_plan {
  std::unique_ptr<TcBatch> b;
};

extern "C" int clc_poisson_sht_batch(clc_ctx* ctx, const double* const* kappa, int nplanes, int nside, int lmax,
                                     int precision, double* const* psi, const clc_derivs* out) {
  if (!ctx) return CLC_EINVAL;
  if (!kappa || nplanes < 1 || !valid_nside(nside) || nside > 4096 || lmax < 1 || lmax > 4 * nside)
    return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: bad arguments");
  for (int i = 0; i < nplanes; ++i)
    if (!kappa[i]) return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: null kappa plane");
  if (precision != CLC_FP64 && precision != CLC_MIXED)
    return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: precision must be CLC_FP64 or CLC_MIXED");
  cudaSetDevice(ctx->device);
  if (precision == CLC_FP64) {
    for (int i = 0; i < nplanes; ++i) {
      const int rc =
          clc_poisson_sht(ctx, kappa[i], nside, lmax, CLC_FP64, psi ? psi[i] : nullptr, out ? &out[i] : nullptr);
      if (rc) return rc;
    }
    return CLC_OK;
  }
  if (nside < 64) return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: CLC_MIXED needs nside >= 64");
  if (!psi && !out) return CLC_OK;
  const int per = tc_class_limit(out != nullptr);
  for (int i0 = 0; i0 < nplanes; i0 += per) {
    const int P = std::min(per, nplanes - i0);
    const int rc = poisson_sht_tc(ctx, kappa + i0, P, nside, lmax, psi ? psi + i0 : nullptr, out ? out + i0 : nullptr);
    if (rc) return rc;
  }
  return CLC_OK;
}

extern "C" int clc_sht_plan_create(clc_ctx* ctx, int nplanes, const int* nside, const int* lmax, int derivatives,
                                   int flags, clc_sht_plan** plan) {
  if (!ctx) return CLC_EINVAL;
  if (!plan || !nside || !lmax || nplanes < 1) return set_err(ctx, CLC_EINVAL, "clc_sht_plan_create: bad arguments");
  *plan = nullptr;
  cudaSetDevice(ctx->device);
  auto p = std::make_unique<clc_sht_plan>();
  p->b = std::make_unique<TcBatch>();
  const int rc = tc_batch_build(ctx, nplanes, nside, lmax, derivatives ? 1 : 0, p->b.get());
  if (rc) return rc;
  p->b->use_graph = (flags & CLC_PLAN_GRAPH) != 0;
  p->b->tune = (flags & CLC_PLAN_TUNE) != 0;
  *plan = p.release();
  return CLC_OK;
}

extern "C" int clc_sht_plan_execute(clc_sht_plan* plan, const double* const* kappa, double* const* psi,
                                    const clc_derivs* out) {
  if (!plan || !plan->b) return CLC_EINVAL;
  clc_ctx* ctx = plan->b->ctx;
  if (!kappa) return set_err(ctx, CLC_EINVAL, "clc_sht_plan_execute: kappa is NULL");
  if (!psi && !out) return CLC_OK;
  cudaSetDevice(ctx->device);
  return tc_batch_execute(plan->b.get(), kappa, psi, out);
}

extern "C" int clc_sht_plan_info(const clc_sht_plan* plan, int* shape, double* stage_ms, size_t* device_bytes) {
  if (!plan || !plan->b) return CLC_EINVAL;
  const TcBatch& B = *plan->b;
  if (shape) {
    shape[0] = B.launch.an_stages;
    shape[1] = B.launch.an_ctas;
    shape[2] = B.launch.sy_stages;
    shape[3] = B.launch.sy_ctas;
    shape[4] = B.launch.fft_ctas;
  }
  if (stage_ms)
    for (int s = 0; s < 6; ++s) stage_ms[s] = B.stage_ms[s];
  if (device_bytes) {
    size_t t = B.work_bytes;
    for (auto& T : B.tabs) t += T->bytes();
    *device_bytes = t;
  }
  return CLC_OK;
}

extern "C" int clc_sht_plan_destroy(clc_sht_plan* plan) {
  if (!plan) return CLC_EINVAL;
  if (plan->b && plan->b->ctx) cudaStreamSynchronize(plan->b->ctx->stream);
  delete plan;
  return CLC_OK;
}
