// Batch plans: many resolvent problems of uneven size (grids, k, shifts) as
// one CUDA graph.  Frequencies are independent problems (Sec. III.B sweeps the
// frequency; Sec. III.A factors once per frequency), so a plan
//   - groups the problems by operator: one batched block factorisation per
//     group over its shifts (the kernels of factor.cu take F problems),
//   - splits every group by k into views that share the group's factors and
//     run Algorithm 1 (sketch, QR, adjoint solve, small SVD, recovery) on
//     their shifts,
//   - records the data-dependent host decisions of an eager calibration run
//     (refinement corrections per solve, shifted CholeskyQR per QR), replays
//     the launch sequence under stream capture with the groups spread over
//     concurrent stream lanes, and instantiates the captured graph: one
//     cudaGraphLaunch runs the whole batch,
//   - optionally tunes the schedule on the device: the trailing-update kernel
//     of each group (128 x 64 tensor-core tiles or 64 x 64 CUDA-core tiles),
//     the K-split of each view's tensor-core sweep, and the number of lanes,
//     each by timing the candidates.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "rr_internal.cuh"

namespace {

struct BView {
  rr_factors* fa = nullptr;  // view over the group's factors
  int k = 0;
  std::vector<int> probs;    // problem indices, in view order
  std::vector<uint64_t> seeds;
  double2* V = nullptr;      // staging [nv][N][k]
  double2* U = nullptr;
  double* sig = nullptr;     // [nv][k]
  double* sh = nullptr;
  std::vector<double> rec_rel;  // recorded final residual per logged solve
  int ks = 0;                // tuned K-split (0 = built-in)
};

struct BGroup {
  rr_operator* op = nullptr;
  rr_factors* fa = nullptr;  // parent factors over the group's shifts
  double* phi = nullptr;     // device [N] (Eq. 9) or null
  std::vector<int> probs;    // problem indices in shift order (sorted by k)
  std::vector<BView> views;
  double cost = 0.0;         // estimated work, for lane assignment
  int lane = 0;
};

struct GuardDev {
  int prev = -1;
  explicit GuardDev(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~GuardDev() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename P>
rr_status balloc(P** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_status(e, "rr_batch_create: cudaMalloc");
  return RR_OK;
}

rr_status berr(rr_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

}  // namespace

struct rr_batch {
  int device = 0;
  rr_precision prec = RR_FP32;
  rr_batch_opts opts{};
  std::vector<rr_problem> probs;
  std::vector<BGroup> groups;
  cudaStream_t cs = nullptr;            // capture origin and calibration stream
  std::vector<cudaStream_t> lanes;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  rr_batch_desc desc{};
};

namespace {

void drop_graph(rr_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

rr_status ensure_lanes(rr_batch* B, int L) {
  while ((int)B->lanes.size() < L) {
    cudaStream_t s;
    cudaEvent_t e;
    RR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    B->lanes.push_back(s);
    RR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B->ev_join.push_back(e);
  }
  return RR_OK;
}

// Longest-processing-time assignment of the groups to L lanes.
void assign_lanes(rr_batch* B, int L) {
  std::vector<int> order(B->groups.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return B->groups[a].cost > B->groups[b].cost; });
  std::vector<double> load(L, 0.0);
  for (int g : order) {
    int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    B->groups[g].lane = l;
    load[l] += B->groups[g].cost;
  }
}

// Algorithm 1 on one view (sketch, then modes), then the per-problem copies
// of the staged results to the caller's buffers.
rr_status run_view(rr_batch* B, BGroup& G, BView& v, rr_info* info) {
  rr_factors* fa = v.fa;
  const int N = G.op->d.n, k = v.k;
  const double tol = B->opts.refine_tol;
  const int maxit = B->opts.max_refine;
  rr_info i1{}, i2{};
  rr_status s = rr_sketch_ex(fa, k, v.seeds.data(), G.phi, nullptr, tol, maxit, v.V, v.sh,
                             info ? &i1 : nullptr);
  rr_status conv = RR_OK;
  if (s == RR_ERR_NOCONV) conv = s; else if (s != RR_OK) return s;
  s = rr_modes(fa, k, v.V, v.U, v.sig, 0, tol, maxit, info ? &i2 : nullptr);
  if (s == RR_ERR_NOCONV) conv = s; else if (s != RR_OK) return s;
  if (info) {
    info->refine_iters = std::max({info->refine_iters, i1.refine_iters, i2.refine_iters});
    info->refine_residual = std::max({info->refine_residual, i1.refine_residual, i2.refine_residual});
    info->cqr_cond = std::max({info->cqr_cond, i1.cqr_cond, i2.cqr_cond});
    info->cqr_shifted |= i1.cqr_shifted | i2.cqr_shifted;
    info->refine_stagnated |= i1.refine_stagnated | i2.refine_stagnated;
    info->first_residual = std::max({info->first_residual, i1.first_residual, i2.first_residual});
    info->problem_solves += i1.problem_solves + i2.problem_solves;
  }
  cudaStream_t st = fa->stream;
  const size_t vb = (size_t)N * k * sizeof(double2), sb = (size_t)k * sizeof(double);
  for (size_t j = 0; j < v.probs.size(); ++j) {
    const rr_problem& p = B->probs[v.probs[j]];
    RR_CUDA(cudaMemcpyAsync(p.V, v.V + j * (size_t)N * k, vb, cudaMemcpyDeviceToDevice, st));
    RR_CUDA(cudaMemcpyAsync(p.U, v.U + j * (size_t)N * k, vb, cudaMemcpyDeviceToDevice, st));
    RR_CUDA(cudaMemcpyAsync(p.sigma, v.sig + j * k, sb, cudaMemcpyDeviceToDevice, st));
    if (p.sigma_halko)
      RR_CUDA(cudaMemcpyAsync(p.sigma_halko, v.sh + j * k, sb, cudaMemcpyDeviceToDevice, st));
  }
  return conv;
}

// Eager calibration run of every view, recording the host decisions.
rr_status record(rr_batch* B) {
  for (auto& G : B->groups)
    for (auto& v : G.views) {
      v.fa->sched_mode = SCHED_RECORD;
      v.fa->sched->clear();
      v.fa->chk_need = 0;
      v.fa->tune_ks = v.ks;
      rr_info info{};
      rr_status s = run_view(B, G, v, &info);
      v.fa->sched_mode = SCHED_EAGER;
      if (s != RR_OK && s != RR_ERR_NOCONV) return s;
      RR_CUDA(cudaStreamSynchronize(v.fa->stream));
      cudaFree(v.fa->chk);
      v.fa->chk = nullptr;
      if ((s = balloc(&v.fa->chk, v.fa->chk_need)) != RR_OK) return s;
      v.fa->chk_cap = v.fa->chk_need;
      v.rec_rel.clear();
    }
  return RR_OK;
}

// Capture the whole batch on L lanes into B->graph and instantiate it.
rr_status capture(rr_batch* B, int L) {
  drop_graph(B);
  rr_status s = ensure_lanes(B, L);
  if (s != RR_OK) return s;
  assign_lanes(B, L);
  std::vector<int> order(B->groups.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return B->groups[a].cost > B->groups[b].cost; });
  // no profiling events or launch counts while recording (the graph's
  // kernels are counted per launch instead)
  ProfSuspend quiet;
  RR_CUDA(cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeRelaxed));
  auto body = [&]() -> rr_status {
    RR_CUDA(cudaEventRecord(B->ev_fork, B->cs));
    for (int l = 0; l < L; ++l) RR_CUDA(cudaStreamWaitEvent(B->lanes[l], B->ev_fork, 0));
    for (int gi : order) {
      BGroup& G = B->groups[gi];
      cudaStream_t st = B->lanes[G.lane];
      G.fa->stream = st;
      rr_status r = factor_async(G.fa);
      if (r != RR_OK) return r;
      for (auto& v : G.views) {
        v.fa->stream = st;
        v.fa->tune_ks = v.ks;
        v.fa->sched_mode = SCHED_REPLAY;
        v.fa->sched_pos = 0;
        v.fa->chk_off = 0;
        v.fa->chk_desc->clear();
        r = run_view(B, G, v, nullptr);
        v.fa->sched_mode = SCHED_EAGER;
        if (r != RR_OK) return r;
        if (v.fa->sched_pos != v.fa->sched->size())
          return berr(RR_ERR_ARG, "rr_batch: replay consumed a different schedule");
      }
    }
    for (int l = 0; l < L; ++l) {
      RR_CUDA(cudaEventRecord(B->ev_join[l], B->lanes[l]));
      RR_CUDA(cudaStreamWaitEvent(B->cs, B->ev_join[l], 0));
    }
    return RR_OK;
  };
  s = body();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->cs, &g);
  if (s != RR_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return s;
  }
  if (e != cudaSuccess) return cuda_status(e, "rr_batch: stream capture");
  B->graph = g;
  RR_CUDA(cudaGraphInstantiate(&B->exec, g, 0));
  size_t n = 0;
  RR_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  RR_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  int kn = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
  }
  B->desc.graph_nodes = (int)n;
  B->desc.kernel_nodes = kn;
  B->desc.lanes = L;
  return RR_OK;
}

// Status and info of the last graph run from the factor flags and the views'
// check logs (stream already synchronised).
rr_status inspect(rr_batch* B, rr_info* info) {
  rr_status worst = RR_OK;
  if (info) *info = rr_info{};
  for (auto& G : B->groups) {
    rr_status s = factor_flags(G.fa);
    if (s != RR_OK) return s;
    for (auto& v : G.views) {
      if ((s = factor_flags(v.fa)) != RR_OK) return s;
      std::vector<char> log(v.fa->chk_off);
      if (!log.empty())
        RR_CUDA(cudaMemcpy(log.data(), v.fa->chk, log.size(), cudaMemcpyDeviceToHost));
      const auto& d = *v.fa->chk_desc;
      size_t nsolve = 0;
      for (size_t t = 0; t + 3 <= d.size(); t += 3) {
        const long long kind = d[t], off = d[t + 1], cnt = d[t + 2];
        if (kind == CHK_SOLVE) {
          const double* bn = reinterpret_cast<const double*>(log.data() + off);
          const double* rn = bn + cnt;
          double rel = 0.0;
          for (long long e = 0; e < cnt; ++e) {
            double r = bn[e] > 0.0 ? rn[e] / bn[e] : rn[e];
            if (!(r == r)) r = INFINITY;
            rel = std::max(rel, r);
          }
          // the recorded run fixes the accuracy this schedule reaches; a
          // residual well above both it and the tolerance means the inputs
          // (new shifts) need more corrections than were recorded
          if (nsolve >= v.rec_rel.size()) v.rec_rel.push_back(rel);
          const double bar = std::max(B->opts.refine_tol, 4.0 * v.rec_rel[nsolve]);
          if (rel > bar && worst == RR_OK) {
            set_error("rr_batch_run: refinement residual above the tolerance for the recorded "
                      "schedule (rebuild the plan for these shifts)");
            worst = RR_ERR_NOCONV;
          }
          ++nsolve;
          if (info) info->refine_residual = std::max(info->refine_residual, rel);
        } else {
          const int* bad = reinterpret_cast<const int*>(log.data() + off);
          const double* cond = reinterpret_cast<const double*>(log.data() + off + cnt * sizeof(double));
          for (long long f = 0; f < cnt; ++f) {
            if (bad[f]) return berr(RR_ERR_RANK, "rr_batch_run: CholeskyQR breakdown");
            if (info) info->cqr_cond = std::max(info->cqr_cond, cond[f]);
          }
        }
      }
      if (info)
        for (size_t t = 0; t < v.fa->sched->size(); ++t)
          info->refine_iters = std::max(info->refine_iters, (*v.fa->sched)[t]);
    }
  }
  return worst;
}

rr_status launch_and_time(rr_batch* B, float* ms) {
  cudaEvent_t e0, e1;
  RR_CUDA(cudaEventCreate(&e0));
  RR_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, B->cs);
  cudaError_t e = cudaGraphLaunch(B->exec, B->cs);
  cudaEventRecord(e1, B->cs);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_status(e, "rr_batch: graph launch");
  prof_count(B->desc.kernel_nodes);
  return RR_OK;
}

float time_factor_cols(rr_factors* fa, int cols) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return INFINITY;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return INFINITY; }
  fa->factor_cols = cols;
  float ms = INFINITY;
  if (factor_async(fa) == RR_OK) {  // warm-up
    cudaEventRecord(e0, fa->stream);
    rr_status s = factor_async(fa);
    cudaEventRecord(e1, fa->stream);
    if (s == RR_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaStreamSynchronize(fa->stream);
  fa->factor_cols = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

rr_status tune(rr_batch* B) {
  // trailing-update tile shape per group, on the first columns
  for (auto& G : B->groups) {
    const OpDev& d = G.op->d;
    if (!tc_prec(B->prec) || d.b < 128 || d.b % 8 != 0) continue;
    const int cols = std::min(d.nx, 6);
    G.fa->tune_update = 0;
    const float t_tc = time_factor_cols(G.fa, cols);
    G.fa->tune_update = 1;
    const float t_cc = time_factor_cols(G.fa, cols);
    G.fa->tune_update = t_cc < t_tc ? 1 : 0;
    // the timing runs overwrote the first columns: refactor with the choice
    rr_status s = factor_async(G.fa);
    if (s != RR_OK) return s;
    RR_CUDA(cudaStreamSynchronize(G.fa->stream));
    if ((s = factor_flags(G.fa)) != RR_OK) return s;
  }
  // K-split of each view's tensor-core sweep
  for (auto& G : B->groups)
    for (auto& v : G.views) {
      if (!sweep_tc2_ok(v.fa, v.k)) continue;
      float best = INFINITY;
      int best_ks = 0;
      for (int ks = 0; ks <= 4; ++ks) {
        v.fa->tune_ks = ks;
        float ms = INFINITY;
        rr_status s = time_solve(v.fa, v.k, &ms);
        if (s != RR_OK) return s;
        if (ms < best * 0.98f) { best = ms; best_ks = ks; }
      }
      v.ks = best_ks;
      v.fa->tune_ks = best_ks;
    }
  return RR_OK;
}

}  // namespace

extern "C" rr_status rr_batch_destroy(rr_batch* B) {
  if (!B) return RR_OK;
  GuardDev guard(B->device);
  if (B->cs) cudaStreamSynchronize(B->cs);
  for (auto s : B->lanes) cudaStreamSynchronize(s);
  drop_graph(B);
  for (auto& G : B->groups) {
    for (auto& v : G.views) {
      rr_destroy_factors(v.fa);
      cudaFree(v.V);
      cudaFree(v.U);
      cudaFree(v.sig);
      cudaFree(v.sh);
    }
    rr_destroy_factors(G.fa);
    cudaFree(G.phi);
  }
  for (auto s : B->lanes) cudaStreamDestroy(s);
  for (auto e : B->ev_join) cudaEventDestroy(e);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->cs) cudaStreamDestroy(B->cs);
  delete B;
  return RR_OK;
}

extern "C" rr_status rr_batch_create(int nprob, const rr_problem* probs, rr_precision prec,
                                     const rr_batch_opts* opts, rr_batch** out) {
  if (!out) return berr(RR_ERR_ARG, "rr_batch_create: null out");
  *out = nullptr;
  if (nprob < 1 || !probs) return berr(RR_ERR_ARG, "rr_batch_create: need at least one problem");
  if (prec != RR_FP64 && prec != RR_FP32 && prec != RR_FP32_SIMT && prec != RR_FP32_BF16X3 &&
      prec != RR_FP32_BF16X6)
    return berr(RR_ERR_ARG, "rr_batch_create: unknown precision");
  rr_batch_opts o{1, 1e-10, 10, 0, 0};
  if (opts) o = *opts;
  if (o.max_refine < 0) return berr(RR_ERR_ARG, "rr_batch_create: max_refine must be >= 0");
  if (o.lanes < 0 || o.lanes > 64) return berr(RR_ERR_ARG, "rr_batch_create: lanes must be in [0, 64]");
  const int device = probs[0].op ? probs[0].op->d.device : 0;
  for (int i = 0; i < nprob; ++i) {
    const rr_problem& p = probs[i];
    if (!p.op || !p.V || !p.U || !p.sigma)
      return berr(RR_ERR_ARG, "rr_batch_create: problem " + std::to_string(i) + " has a null pointer");
    if (p.op->d.device != device)
      return berr(RR_ERR_ARG, "rr_batch_create: all operators must be on one device");
    if (p.k < 1 || p.k > 64 || p.k > p.op->d.n)
      return berr(RR_ERR_ARG, "rr_batch_create: problem " + std::to_string(i) +
                                  " needs k in [1, min(64, N)]");
    if (!std::isfinite(p.s_re) || !std::isfinite(p.s_im))
      return berr(RR_ERR_ARG, "rr_batch_create: shifts must be finite");
  }
  const auto t0 = std::chrono::steady_clock::now();
  GuardDev guard(device);
  rr_batch* B = new rr_batch();
  B->device = device;
  B->prec = prec;
  B->opts = o;
  B->probs.assign(probs, probs + nprob);
  auto fail = [&](rr_status s) {
    rr_batch_destroy(B);
    return s;
  };
  {
    cudaError_t e = cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_status(e, "rr_batch_create: stream"));
  }
  // groups by operator (first appearance order); problems sorted by k inside
  for (int i = 0; i < nprob; ++i) {
    auto it = std::find_if(B->groups.begin(), B->groups.end(),
                           [&](const BGroup& g) { return g.op == probs[i].op; });
    if (it == B->groups.end()) {
      B->groups.emplace_back();
      B->groups.back().op = probs[i].op;
      it = B->groups.end() - 1;
    }
    it->probs.push_back(i);
  }
  rr_status s;
  for (auto& G : B->groups) {
    std::stable_sort(G.probs.begin(), G.probs.end(),
                     [&](int a, int b) { return probs[a].k < probs[b].k; });
    const OpDev& d = G.op->d;
    const int ng = (int)G.probs.size();
    std::vector<double> sh(2 * ng);
    for (int j = 0; j < ng; ++j) {
      sh[2 * j] = probs[G.probs[j]].s_re;
      sh[2 * j + 1] = probs[G.probs[j]].s_im;
    }
    // calibration factorisation (eager; also validates the shifts)
    if ((s = rr_factor(G.op, ng, sh.data(), prec, B->cs, &G.fa)) != RR_OK) {
      if (G.fa) { rr_destroy_factors(G.fa); G.fa = nullptr; }
      return fail(s);
    }
    G.cost = (double)ng * d.nx * (double)d.b * d.b * d.b;
    if (o.use_phi) {
      if ((s = balloc(&G.phi, (size_t)d.n * sizeof(double))) != RR_OK) return fail(s);
      if ((s = launch_phi(d, G.phi, B->cs)) != RR_OK) return fail(s);
    }
    // views: runs of equal k
    for (int j0 = 0; j0 < ng;) {
      int j1 = j0;
      const int k = probs[G.probs[j0]].k;
      while (j1 < ng && probs[G.probs[j1]].k == k) ++j1;
      G.views.emplace_back();
      BView& v = G.views.back();
      v.k = k;
      v.probs.assign(G.probs.begin() + j0, G.probs.begin() + j1);
      for (int p : v.probs) v.seeds.push_back(probs[p].seed);
      const int nv = j1 - j0;
      if ((s = factors_view(G.fa, j0, nv, B->cs, &v.fa)) != RR_OK) return fail(s);
      if ((s = factors_reserve(v.fa, k)) != RR_OK) return fail(s);
      const size_t vb = (size_t)nv * d.n * k * sizeof(double2);
      if ((s = balloc(&v.V, vb)) != RR_OK) return fail(s);
      if ((s = balloc(&v.U, vb)) != RR_OK) return fail(s);
      if ((s = balloc(&v.sig, (size_t)nv * k * sizeof(double))) != RR_OK) return fail(s);
      if ((s = balloc(&v.sh, (size_t)nv * k * sizeof(double))) != RR_OK) return fail(s);
      G.cost += 6.0 * nv * d.nx * (double)d.b * d.b * k;
      j0 = j1;
    }
  }
  {
    cudaError_t e = cudaStreamSynchronize(B->cs);
    if (e != cudaSuccess) return fail(cuda_status(e, "rr_batch_create"));
  }
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point a) {
    return std::chrono::duration<double, std::milli>(clk::now() - a).count();
  };
  double calib_ms = ms_since(t0), tune_ms = 0.0;
  auto t1 = clk::now();
  if (o.tune && (s = tune(B)) != RR_OK) return fail(s);
  tune_ms += ms_since(t1);
  t1 = clk::now();
  if ((s = record(B)) != RR_OK) return fail(s);
  calib_ms += ms_since(t1);
  t1 = clk::now();
  // lanes: the given count, the candidates the tuner times, or min(groups, 4)
  const int ngroups = (int)B->groups.size();
  std::vector<int> cands;
  if (o.lanes > 0) {
    cands.push_back(std::min(o.lanes, ngroups));
  } else if (o.tune) {
    // one lane (fully serial groups) is timed only for tiny plans
    for (int L : {1, 2, 4, 8, ngroups})
      if (L <= ngroups && (L > 1 || ngroups <= 2) &&
          std::find(cands.begin(), cands.end(), L) == cands.end())
        cands.push_back(L);
  } else {
    cands.push_back(std::min(ngroups, 4));
  }
  int bestL = cands[0];
  float best = INFINITY;
  if (cands.size() > 1) {
    for (int L : cands) {
      if ((s = capture(B, L)) != RR_OK) return fail(s);
      // the upload keeps the graph's one-off setup out of the timed launch
      cudaError_t ue = cudaGraphUpload(B->exec, B->cs);
      if (ue != cudaSuccess) return fail(cuda_status(ue, "rr_batch_create: graph upload"));
      float ms = INFINITY;
      if ((s = launch_and_time(B, &ms)) != RR_OK) return fail(s);
      if (ms < best) { best = ms; bestL = L; }
    }
  }
  tune_ms += ms_since(t1);
  t1 = clk::now();
  if ((s = capture(B, bestL)) != RR_OK) return fail(s);
  {
    cudaError_t ue = cudaGraphUpload(B->exec, B->cs);
    if (ue != cudaSuccess) return fail(cuda_status(ue, "rr_batch_create: graph upload"));
  }
  B->desc.capture_ms = ms_since(t1);
  B->desc.calib_ms = calib_ms;
  B->desc.tune_ms = tune_ms;
  // validation run: the graph reproduces the calibration run, and its
  // residuals become the reference the checks of later runs compare with
  {
    cudaError_t e = cudaGraphLaunch(B->exec, B->cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->cs);
    if (e != cudaSuccess) return fail(cuda_status(e, "rr_batch_create: validation run"));
    prof_count(B->desc.kernel_nodes);
    s = inspect(B, nullptr);
    if (s != RR_OK && s != RR_ERR_NOCONV) return fail(s);
  }
  B->desc.groups = ngroups;
  int nviews = 0, ncc = 0;
  for (auto& G : B->groups) {
    nviews += (int)G.views.size();
    ncc += G.fa->tune_update == 1 ? 1 : 0;
  }
  B->desc.views = nviews;
  B->desc.cuda_core_updates = ncc;
  B->desc.tuned_ms = std::isfinite(best) ? best : 0.0;
  B->desc.plan_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = B;
  return RR_OK;
}

extern "C" rr_status rr_batch_run(rr_batch* B, void* stream, rr_info* info) {
  if (!B || !B->exec) return berr(RR_ERR_ARG, "rr_batch_run: null plan");
  GuardDev guard(B->device);
  cudaStream_t st = stream ? reinterpret_cast<cudaStream_t>(stream) : B->cs;
  RR_CUDA(cudaGraphLaunch(B->exec, st));
  RR_CUDA(cudaStreamSynchronize(st));
  prof_count(B->desc.kernel_nodes);
  return inspect(B, info);
}

extern "C" rr_status rr_batch_set_shifts(rr_batch* B, const double* shifts) {
  if (!B || !shifts) return berr(RR_ERR_ARG, "rr_batch_set_shifts: null argument");
  const int n = (int)B->probs.size();
  for (int i = 0; i < 2 * n; ++i)
    if (!std::isfinite(shifts[i])) return berr(RR_ERR_ARG, "rr_batch_set_shifts: shifts must be finite");
  GuardDev guard(B->device);
  RR_CUDA(cudaStreamSynchronize(B->cs));
  for (auto l : B->lanes) RR_CUDA(cudaStreamSynchronize(l));
  for (int i = 0; i < n; ++i) {
    B->probs[i].s_re = shifts[2 * i];
    B->probs[i].s_im = shifts[2 * i + 1];
  }
  for (auto& G : B->groups) {
    const int ng = (int)G.probs.size();
    for (int j = 0; j < ng; ++j)
      G.fa->shifts_h[j] = make_double2(B->probs[G.probs[j]].s_re, B->probs[G.probs[j]].s_im);
    RR_CUDA(cudaMemcpy(G.fa->shifts, G.fa->shifts_h, ng * sizeof(double2), cudaMemcpyHostToDevice));
    int j0 = 0;
    for (auto& v : G.views) {
      for (int j = 0; j < v.fa->F; ++j) v.fa->shifts_h[j] = G.fa->shifts_h[j0 + j];
      j0 += v.fa->F;
    }
  }
  return RR_OK;
}

extern "C" rr_status rr_batch_describe(const rr_batch* B, rr_batch_desc* d) {
  if (!B || !d) return berr(RR_ERR_ARG, "rr_batch_describe: null argument");
  *d = B->desc;
  return RR_OK;
}
