// C ABI of librr: operator and factor handles, and the host orchestration of
// Algorithm 1 (Sec. II.B) over the device kernels.  Every step of the path
// runs on the GPU; the host only sequences launches and, for the iterative
// refinement of the FP32 factors, reads back residual norms.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rr_internal.cuh"

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

rr_status cuda_status(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? RR_ERR_NOMEM : RR_ERR_CUDA;
}

static rr_status arg_error(const std::string& msg) {
  g_err = msg;
  return RR_ERR_ARG;
}

int num_sms(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 152;
  if (cached[device] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
      v = 152;
    cached[device] = v;
  }
  return cached[device];
}

extern "C" const char* rr_last_error(void) { return g_err.c_str(); }

extern "C" const char* rr_status_string(rr_status s) {
  switch (s) {
    case RR_OK: return "ok";
    case RR_ERR_ARG: return "invalid argument";
    case RR_ERR_NOMEM: return "out of device memory";
    case RR_ERR_SINGULAR: return "singular pivot";
    case RR_ERR_NOCONV: return "refinement did not converge";
    case RR_ERR_RANK: return "CholeskyQR breakdown";
    case RR_ERR_TIMEOUT: return "device wait timed out";
    case RR_ERR_CUDA: return "CUDA error";
    case RR_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename P>
rr_status dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[128];
    snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    g_err = buf;
    return RR_ERR_NOMEM;
  }
  return RR_OK;
}

// Sketch workspace carved out of one allocation.
struct Work {
  double2 *W1, *W2, *W3, *R64;  // [F][N][k] FP64
  void *L1, *L2, *L3;           // [F][N][k] factor precision
  double2 *G, *R1, *R1i, *R2, *R2i, *Rt, *Ul, *Vr, *Rd;  // [F][k][k]
  double2* part;                // gram partials
  double* dpart;                // norm / max partials
  double *sig, *cond, *bn, *rn; // [F][k] or [F]
  int *bad, *rank, *sweeps;
  double2* phase;
  uint64_t* seeds;
  double* featbar;              // [nx*ny][18] gradient scratch
  int nblk_gram, nblk_col;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Compute the layout (or carve it when base != nullptr); returns total bytes.
size_t carve(rr_factors* fa, int k, char* base, Work* w) {
  const int F = fa->F, N = fa->op->d.n;
  const size_t vec64 = (size_t)F * N * k * sizeof(double2);
  const size_t veclo = (size_t)F * N * k * fa->csz;
  const size_t small = (size_t)F * k * k * sizeof(double2);
  int nblk_gram = std::max(1, std::min(N / 64, std::max(1, 2 * num_sms(fa->op->d.device) / F)));
  int nblk_col = nblk_gram;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return base ? base + o : nullptr;
  };
  Work t;
  t.W1 = (double2*)take(vec64);
  t.W2 = (double2*)take(vec64);
  t.W3 = (double2*)take(vec64);
  t.R64 = (double2*)take(vec64);
  t.L1 = take(veclo);
  t.L2 = take(veclo);
  t.L3 = take(veclo);
  t.G = (double2*)take(small);
  t.R1 = (double2*)take(small);
  t.R1i = (double2*)take(small);
  t.R2 = (double2*)take(small);
  t.R2i = (double2*)take(small);
  t.Rt = (double2*)take(small);
  t.Ul = (double2*)take(small);
  t.Vr = (double2*)take(small);
  t.Rd = (double2*)take(small);
  t.part = (double2*)take((size_t)F * nblk_gram * k * k * sizeof(double2));
  t.dpart = (double*)take((size_t)F * nblk_col * k * (sizeof(double) + sizeof(int)));
  t.sig = (double*)take((size_t)F * k * sizeof(double));
  t.cond = (double*)take((size_t)F * sizeof(double));
  t.bn = (double*)take((size_t)F * k * sizeof(double));
  t.rn = (double*)take((size_t)F * k * sizeof(double));
  t.bad = (int*)take((size_t)F * sizeof(int));
  t.rank = (int*)take((size_t)F * k * sizeof(int));
  t.sweeps = (int*)take((size_t)F * sizeof(int));
  t.phase = (double2*)take((size_t)F * k * sizeof(double2));
  t.seeds = (uint64_t*)take((size_t)F * sizeof(uint64_t));
  t.featbar = (double*)take((size_t)fa->op->d.nx * fa->op->d.ny * 18 * sizeof(double));
  t.nblk_gram = nblk_gram;
  t.nblk_col = nblk_col;
  if (w) *w = t;
  return off;
}

rr_status get_work(rr_factors* fa, int k, Work* w) {
  if (k > fa->kmax || fa->ws == nullptr) {
    if (fa->ws) {
      cudaStreamSynchronize(fa->stream);
      cudaFree(fa->ws);
      fa->ws = nullptr;
    }
    size_t bytes = carve(fa, k, nullptr, nullptr);
    rr_status s = dalloc(reinterpret_cast<char**>(&fa->ws), bytes);
    if (s != RR_OK) return s;
    fa->ws_bytes = bytes;
    fa->kmax = k;
  }
  carve(fa, k, reinterpret_cast<char*>(fa->ws), w);
  return RR_OK;
}

void info_reset(rr_info* info) {
  if (!info) return;
  info->refine_iters = 0;
  info->refine_residual = 0.0;
  info->cqr_cond = 0.0;
  info->cqr_shifted = 0;
  info->refine_stagnated = 0;
  info->first_residual = 0.0;
  info->problem_solves = 0;
}

// x = A^{-1} b (or A^{-H} b) in FP64 [F][N][k], b != x, with FP64 iterative
// refinement: x <- x + solve(b - A x) until every column's relative residual
// is at most tol (tol <= 0: one solve, residual reported only when info).
rr_status solve_refined(rr_factors* fa, int k, int adjoint, const double2* b, double2* x,
                        double tol, int maxit, Work& w, rr_info* info) {
  const OpDev& d = fa->op->d;
  const int F = fa->F;
  const size_t nel = (size_t)F * d.n * k;
  cudaStream_t st = fa->stream;
  const bool lo = fa->prec != RR_FP64;
  rr_status s;
  // first solve
  if (!lo) {
    if ((s = launch_solve_lo(fa, k, adjoint, b, x, w.L3)) != RR_OK) return s;
  } else {
    if ((s = launch_convert_d2f(nel, b, (float2*)w.L1, st)) != RR_OK) return s;
    if ((s = launch_solve_lo(fa, k, adjoint, w.L1, w.L2, w.L3)) != RR_OK) return s;
    if ((s = launch_convert_f2d(nel, (const float2*)w.L2, x, 0, st)) != RR_OK) return s;
  }
  if (info) info->problem_solves += F;
  const bool check = lo || info != nullptr || tol > 0.0 || fa->sched_mode != SCHED_EAGER;
  if (!check) return RR_OK;
  if ((s = launch_colnorm2(F, d.n, k, b, w.dpart, w.nblk_col, w.bn, st)) != RR_OK) return s;
  if (fa->sched_mode == SCHED_REPLAY) {
    // the recorded number of corrections, no host reads; the final residual
    // and right-hand-side norms go to the check log
    if (fa->sched_pos >= fa->sched->size()) {
      g_err = "graph schedule exhausted (launch sequence differs from the recorded one)";
      return RR_ERR_ARG;
    }
    const int nit = (*fa->sched)[fa->sched_pos++];
    if (info) info->problem_solves += (long long)nit * F;
    for (int t = 0; t < nit; ++t) {
      if ((s = launch_residual(d, F, fa->shifts, k, adjoint, b, x, w.R64, st)) != RR_OK) return s;
      if (!lo) {
        if ((s = launch_solve_lo(fa, k, adjoint, w.R64, w.L2, w.L3)) != RR_OK) return s;
        if ((s = launch_axpy(nel, (const double2*)w.L2, x, st)) != RR_OK) return s;
      } else {
        if ((s = launch_convert_d2f(nel, w.R64, (float2*)w.L1, st)) != RR_OK) return s;
        if ((s = launch_solve_lo(fa, k, adjoint, w.L1, w.L2, w.L3)) != RR_OK) return s;
        if ((s = launch_convert_f2d(nel, (const float2*)w.L2, x, 1, st)) != RR_OK) return s;
      }
    }
    if ((s = launch_residual(d, F, fa->shifts, k, adjoint, b, x, w.R64, st)) != RR_OK) return s;
    if ((s = launch_colnorm2(F, d.n, k, w.R64, w.dpart, w.nblk_col, w.rn, st)) != RR_OK) return s;
    const size_t nb = (size_t)F * k * sizeof(double);
    if (fa->chk_off + 2 * nb > fa->chk_cap) {
      g_err = "graph check log too small";
      return RR_ERR_ARG;
    }
    RR_CUDA(cudaMemcpyAsync(fa->chk + fa->chk_off, w.bn, nb, cudaMemcpyDeviceToDevice, st));
    RR_CUDA(cudaMemcpyAsync(fa->chk + fa->chk_off + nb, w.rn, nb, cudaMemcpyDeviceToDevice, st));
    fa->chk_desc->insert(fa->chk_desc->end(), {CHK_SOLVE, (long long)fa->chk_off, (long long)F * k});
    fa->chk_off += 2 * nb;
    return RR_OK;
  }
  if (fa->sched_mode == SCHED_RECORD) fa->chk_need += 2 * (size_t)F * k * sizeof(double);
  std::vector<double> bn((size_t)F * k), rn((size_t)F * k);
  RR_CUDA(cudaMemcpyAsync(bn.data(), w.bn, bn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  // Eager solves on the split tensor-core sweep refine each problem on its
  // own: a problem leaves the active set once its residual meets tol or a
  // correction no longer halves it, and the corrections and residuals that
  // follow run on the active problems only.  Elsewhere (and when recording a
  // schedule) all problems take every correction until the largest residual
  // meets tol or stops halving.
  const bool per_problem = fa->sched_mode == SCHED_EAGER && lo && sweep_tc2_ok(fa, k);
  struct MapReset {  // the solve path never keeps a subset past this call
    rr_factors* fa;
    ~MapReset() {
      fa->amap = nullptr;
      fa->Fa = 0;
    }
  } map_reset{fa};
  std::vector<double> relf(F, 0.0), prevf(F, INFINITY);
  std::vector<char> active(F, 1);
  std::vector<int> act;  // active problems of the last correction
  bool subset = false;   // residuals on the list in amap_buf
  int it = 0;
  double rel = 0.0, prev = INFINITY;
  int stagnated = 0;
  rr_status result = RR_OK;
  for (;;) {
    const int* amap = subset ? fa->amap_buf : nullptr;
    const int nres = subset ? (int)act.size() : F;
    if ((s = launch_residual(d, nres, fa->shifts, k, adjoint, b, x, w.R64, st, amap)) != RR_OK)
      return s;
    if ((s = launch_colnorm2(nres, d.n, k, w.R64, w.dpart, w.nblk_col, w.rn, st, amap)) != RR_OK)
      return s;
    RR_CUDA(cudaMemcpyAsync(rn.data(), w.rn, rn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    int tc_err = 0;
    RR_CUDA(cudaMemcpyAsync(&tc_err, fa->flag + F, sizeof(int), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (tc_err) {
      // reported once: the flag is cleared so the factors serve later solves
      RR_CUDA(cudaMemsetAsync(fa->flag + F, 0, sizeof(int), st));
      RR_CUDA(cudaStreamSynchronize(st));
      g_err = "a tensor-core sweep kernel timed out in a bounded wait";
      return RR_ERR_TIMEOUT;
    }
    rel = 0.0;
    for (int f = 0; f < F; ++f) {
      if (!subset || active[f]) {
        double rf = 0.0;
        for (int j = 0; j < k; ++j) {
          const size_t e = (size_t)f * k + j;
          double r = bn[e] > 0.0 ? rn[e] / bn[e] : rn[e];
          if (!(r == r)) r = INFINITY;
          rf = std::max(rf, r);
        }
        relf[f] = rf;
      }
      rel = std::max(rel, relf[f]);
    }
    if (it == 0 && info) info->first_residual = std::max(info->first_residual, rel);
    if (tol <= 0.0) break;
    // The FP64 residual itself carries rounding of order u ||A|| ||x||, and
    // where the FP32 factors resolve some directions only to O(1) a
    // correction contracts the residual slowly; refinement goes on while a
    // correction still removes at least a tenth of the residual and stops
    // (stagnated) once it does not: at that point x is as accurate as the
    // floor allows and further sweeps cannot help.
    constexpr double kStagnation = 0.9;
    if (per_problem) {
      act.clear();
      for (int f = 0; f < F; ++f) {
        if (!active[f]) continue;
        if (relf[f] <= tol) {
          active[f] = 0;
        } else if (it > 0 && relf[f] > kStagnation * prevf[f]) {
          active[f] = 0;
          stagnated = 1;
        } else {
          prevf[f] = relf[f];
          act.push_back(f);
        }
      }
      if (act.empty()) break;
    } else {
      if (rel <= tol) break;
      if (it > 0 && rel > kStagnation * prev) {
        stagnated = 1;
        break;
      }
      prev = rel;
    }
    if (it >= maxit) {
      char buf[160];
      snprintf(buf, sizeof buf, "refinement stopped after %d iterations at relative residual %.3e > %.3e",
               it, rel, tol);
      g_err = buf;
      result = RR_ERR_NOCONV;
      break;
    }
    // correction d = solve(r); x += d
    if (info) info->problem_solves += per_problem ? (long long)act.size() : F;
    if (per_problem) {
      const size_t nk = (size_t)d.n * k;
      RR_CUDA(cudaMemcpyAsync(fa->amap_buf, act.data(), act.size() * sizeof(int),
                              cudaMemcpyHostToDevice, st));
      fa->amap = fa->amap_buf;
      fa->Fa = (int)act.size();
      fa->amap_h = act;
      if ((s = launch_convert_d2f_map(fa->Fa, fa->amap, nk, w.R64, (float2*)w.L1, st)) != RR_OK)
        return s;
      if ((s = launch_solve_lo(fa, k, adjoint, w.L1, w.L2, w.L3)) != RR_OK) return s;
      if ((s = launch_convert_f2d_map(fa->Fa, fa->amap, nk, (const float2*)w.L2, x, 1, st)) !=
          RR_OK)
        return s;
      fa->amap = nullptr;
      fa->Fa = 0;
      subset = true;
    } else if (!lo) {
      // FP64 factors: the correction lands in L2 (complex double here)
      if ((s = launch_solve_lo(fa, k, adjoint, w.R64, w.L2, w.L3)) != RR_OK) return s;
      if ((s = launch_axpy(nel, (const double2*)w.L2, x, st)) != RR_OK) return s;
    } else {
      if ((s = launch_convert_d2f(nel, w.R64, (float2*)w.L1, st)) != RR_OK) return s;
      if ((s = launch_solve_lo(fa, k, adjoint, w.L1, w.L2, w.L3)) != RR_OK) return s;
      if ((s = launch_convert_f2d(nel, (const float2*)w.L2, x, 1, st)) != RR_OK) return s;
    }
    ++it;
  }
  if (info) {
    info->refine_iters = std::max(info->refine_iters, it);
    info->refine_residual = std::max(info->refine_residual, rel);
    info->refine_stagnated |= stagnated;
  }
  if (fa->sched_mode == SCHED_RECORD) fa->sched->push_back(it);
  return result;
}

// CholeskyQR2 (shifted CholeskyQR3 on breakdown) of Y in place; R = R2 R1 (R3).
// With defer_rinv, the last pass's multiply is left to the caller: Y holds
// Q R_last (the previous pass's Q) and defer_rinv receives R_last^{-1}, so a
// caller that needs Q S forms it as Y (R_last^{-1} S) in one multiply.
rr_status cholqr2(rr_factors* fa, int k, double2* Y, double2* Rout, Work& w, rr_info* info,
                  double2* defer_rinv = nullptr) {
  const int F = fa->F, N = fa->op->d.n;
  cudaStream_t st = fa->stream;
  rr_status s;
  RR_CUDA(cudaMemsetAsync(w.bad, 0, F * sizeof(int), st));
  if ((s = launch_gram(F, N, k, Y, w.part, w.nblk_gram, w.G, st)) != RR_OK) return s;
  if ((s = launch_cholesky(F, k, w.G, w.R1, w.R1i, w.bad, 0.0, w.cond, st)) != RR_OK) return s;
  const bool replay = fa->sched_mode == SCHED_REPLAY;
  std::vector<int> bad(F);
  std::vector<double> cond(F);
  bool any_bad = false;
  if (replay) {
    if (fa->sched_pos >= fa->sched->size()) {
      g_err = "graph schedule exhausted (launch sequence differs from the recorded one)";
      return RR_ERR_ARG;
    }
    any_bad = (*fa->sched)[fa->sched_pos++] != 0;
  } else {
    RR_CUDA(cudaMemcpyAsync(bad.data(), w.bad, F * sizeof(int), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(cond.data(), w.cond, F * sizeof(double), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    for (int f = 0; f < F; ++f) any_bad |= bad[f] != 0;
    if (fa->sched_mode == SCHED_RECORD) {
      fa->sched->push_back(any_bad ? 1 : 0);
      fa->chk_need += (size_t)F * (sizeof(double) + sizeof(double));
    }
  }
  int passes = 2;
  if (any_bad) {
    // shifted CholeskyQR (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
    // SIAM J. Sci. Comput. 2020): shift 11 (N k + k (k + 1)) u ||Y||^2,
    // with trace(G) >= ||Y||_2^2, then two plain passes.
    const double u = std::ldexp(1.0, -53);
    double shift_rel = 11.0 * ((double)N * k + (double)k * (k + 1)) * u;
    RR_CUDA(cudaMemsetAsync(w.bad, 0, F * sizeof(int), st));
    if ((s = launch_cholesky(F, k, w.G, w.R1, w.R1i, w.bad, shift_rel, w.cond, st)) != RR_OK)
      return s;
    if (info) info->cqr_shifted = 1;
    passes = 3;
  }
  for (int f = 0; f < F; ++f)
    if (info) info->cqr_cond = std::max(info->cqr_cond, cond[f]);
  if ((s = launch_right_mul(F, N, k, Y, w.R1i, Y, st, 1)) != RR_OK) return s;
  RR_CUDA(cudaMemcpyAsync(w.Rt, w.R1, (size_t)F * k * k * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  for (int p = 1; p < passes; ++p) {
    RR_CUDA(cudaMemsetAsync(w.bad, 0, F * sizeof(int), st));
    if ((s = launch_gram(F, N, k, Y, w.part, w.nblk_gram, w.G, st)) != RR_OK) return s;
    if ((s = launch_cholesky(F, k, w.G, w.R2, w.R2i, w.bad, 0.0, nullptr, st)) != RR_OK) return s;
    if (defer_rinv && p + 1 == passes)
      RR_CUDA(cudaMemcpyAsync(defer_rinv, w.R2i, (size_t)F * k * k * sizeof(double2),
                              cudaMemcpyDeviceToDevice, st));
    else if ((s = launch_right_mul(F, N, k, Y, w.R2i, Y, st, 1)) != RR_OK)
      return s;
    if ((s = launch_small_mul(F, k, w.R2, w.Rt, w.R1, st)) != RR_OK) return s;
    RR_CUDA(cudaMemcpyAsync(w.Rt, w.R1, (size_t)F * k * k * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  }
  if (replay) {
    // breakdown flags and the first pass's condition estimate, checked after
    // the graph has run
    const size_t nb = (size_t)F * sizeof(double);
    if (fa->chk_off + 2 * nb > fa->chk_cap) {
      g_err = "graph check log too small";
      return RR_ERR_ARG;
    }
    RR_CUDA(cudaMemcpyAsync(fa->chk + fa->chk_off, w.bad, F * sizeof(int), cudaMemcpyDeviceToDevice, st));
    RR_CUDA(cudaMemcpyAsync(fa->chk + fa->chk_off + nb, w.cond, nb, cudaMemcpyDeviceToDevice, st));
    fa->chk_desc->insert(fa->chk_desc->end(), {CHK_CQR, (long long)fa->chk_off, (long long)F});
    fa->chk_off += 2 * nb;
  } else {
    RR_CUDA(cudaMemcpyAsync(bad.data(), w.bad, F * sizeof(int), cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    for (int f = 0; f < F; ++f)
      if (bad[f]) {
        g_err = "CholeskyQR breakdown: the sketch is numerically rank deficient";
        return RR_ERR_RANK;
      }
  }
  if (Rout)
    RR_CUDA(cudaMemcpyAsync(Rout, w.Rt, (size_t)F * k * k * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  return RR_OK;
}

}  // namespace

// TMA tensor maps over all FP32 factors G [F][nx][b][b] (complex, viewed as
// floats [F*nx][b][2b]): tiles of 128 rows x 16 complex (G) and of 16 rows x
// 128 complex (for G^H).  Used only when b >= 128 and the row pitch is a
// multiple of 16 bytes (b even); otherwise the sweeps use cp.async kernels.
static int encode_factor_maps(rr_factors* fa) {
  const OpDev& d = fa->op->d;
  if (d.b < 128 || (d.b & 1)) return 0;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr) {
      cudaGetLastError();
      return 0;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)2 * d.b, (cuuint64_t)d.b, (cuuint64_t)fa->F * d.nx};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * d.b * 4, (cuuint64_t)2 * d.b * d.b * 4};
  const cuuint32_t boxN[3] = {32, 128, 1}, boxT[3] = {256, 16, 1}, es[3] = {1, 1, 1};
  CUresult r1 = encode(reinterpret_cast<CUtensorMap*>(fa->tmap[0]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                       3, fa->G, dims, strides, boxN, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = encode(reinterpret_cast<CUtensorMap*>(fa->tmap[1]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                       3, fa->G, dims, strides, boxT, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? 1 : 0;
}

// TMA map over the FP32 work matrices M [F][b][b] (complex, viewed as floats
// [F][b][2b]): tiles of 128 rows x 32 complex, the A operand of the
// tensor-core trailing update.  Needs b >= 128 and b % 8 == 0.
static int encode_m_map(rr_factors* fa) {
  const OpDev& d = fa->op->d;
  if (!tc_prec(fa->prec) || d.b < 128 || (d.b & 7)) return 0;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return 0;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[3] = {(cuuint64_t)2 * d.b, (cuuint64_t)d.b, (cuuint64_t)fa->F};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * d.b * 4, (cuuint64_t)2 * d.b * d.b * 4};
  const cuuint32_t box[3] = {64, 128, 1}, es[3] = {1, 1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(fa->tmap[2]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      3, fa->M, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 1 : 0;
}

// TMA maps of the wide factorisation (FP32 factors): chunks of 16 complex
// columns x 128 rows of M (the left operand of the rank-128 update, read in
// place), and tiles of 16 rows x 64 complex of the gathered pivot rows Wbuf
// [F][128][b] (its right operand).
static int encode_wide_maps(rr_factors* fa) {
  const OpDev& d = fa->op->d;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return 0;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint32_t es[3] = {1, 1, 1};
  const cuuint64_t dm[3] = {(cuuint64_t)2 * d.b, (cuuint64_t)d.b, (cuuint64_t)fa->F};
  const cuuint64_t sm[2] = {(cuuint64_t)2 * d.b * 4, (cuuint64_t)2 * d.b * d.b * 4};
  const cuuint32_t boxA[3] = {32, 128, 1}, boxB[3] = {128, 16, 1};
  const cuuint64_t dw[3] = {(cuuint64_t)2 * d.b, 128, (cuuint64_t)fa->F};
  const cuuint64_t sw[2] = {(cuuint64_t)2 * d.b * 4, (cuuint64_t)2 * d.b * 128 * 4};
  CUresult r0 = encode(reinterpret_cast<CUtensorMap*>(fa->wmap[0]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                       3, fa->M, dm, sm, boxA, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r1 = encode(reinterpret_cast<CUtensorMap*>(fa->wmap[1]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                       3, fa->Wbuf, dw, sw, boxB, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return (r0 == CUDA_SUCCESS && r1 == CUDA_SUCCESS) ? 1 : 0;
}

// ----------------------------------------------------------------- operator
extern "C" rr_status rr_create_operator(const rr_grid* g, const rr_baseflow* fl,
                                        const double* weights, int device, rr_operator** out) {
  if (!g || !fl || !out) return arg_error("rr_create_operator: null argument");
  *out = nullptr;
  if (g->kind != RR_ADVDIFF_SCALAR && g->kind != RR_ISO_NS2D && g->kind != RR_ISO_NS2D_KZ)
    return arg_error("rr_create_operator: unknown operator kind");
  const bool ns = g->kind != RR_ADVDIFF_SCALAR;
  if (g->kind == RR_ISO_NS2D_KZ && !std::isfinite(g->kz))
    return arg_error("rr_create_operator: kz must be finite");
  if (g->nx < 3 || g->ny < 3) return arg_error("rr_create_operator: nx and ny must be >= 3");
  const int q = g->kind;
  if (q * g->ny > 1024) return arg_error("rr_create_operator: block size q*ny must be <= 1024");
  if (!(g->re > 0)) return arg_error("rr_create_operator: re must be positive");
  if (ns && !(g->mach > 0))
    return arg_error("rr_create_operator: mach must be positive");
  if (!(g->x1 > g->x0) || !(g->y1 > g->y0)) return arg_error("rr_create_operator: empty domain");
  if (g->sponge_max != 0.0 && !(g->sponge_frac > 0.0 && g->sponge_frac <= 0.5))
    return arg_error("rr_create_operator: sponge_frac must be in (0, 0.5]");
  for (int e = 0; e < 4; ++e)
    if (g->neumann[e] < 0 || g->neumann[e] >= (1 << g->kind))
      return arg_error("rr_create_operator: neumann masks must be bit masks over the q variables");
  if (g->periodic_y && (g->neumann[2] || g->neumann[3]))
    return arg_error("rr_create_operator: a periodic y direction has no y boundary closure");
  if (!fl->u || !fl->v || (ns && !fl->rho))
    return arg_error("rr_create_operator: missing base-flow field");
  const size_t npts = (size_t)g->nx * g->ny;
  const size_t N = npts * q;
  if (N > (size_t)1 << 30) return arg_error("rr_create_operator: too many unknowns");
  if (weights)
    for (size_t n = 0; n < N; ++n)
      if (!(weights[n] > 0.0) || !std::isfinite(weights[n]))
        return arg_error("rr_create_operator: weights must be positive and finite");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    g_err = "rr_create_operator: no CUDA device";
    return RR_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return arg_error("rr_create_operator: bad device ordinal");
  DeviceGuard guard(device);
  rr_operator* op = new rr_operator();
  op->grid = *g;
  OpDev& d = op->d;
  d.kind = g->kind; d.q = q; d.nx = g->nx; d.ny = g->ny; d.b = q * g->ny; d.n = (int)N;
  d.periodic = g->periodic_y ? 1 : 0;
  d.dx = (g->x1 - g->x0) / (g->nx + 1);
  d.dy = d.periodic ? (g->y1 - g->y0) / g->ny : (g->y1 - g->y0) / (g->ny + 1);
  d.device = device;
  d.coef = nullptr; d.coef32 = nullptr; d.wsqrt = nullptr; d.wisqrt = nullptr; d.flow = nullptr;
  d.ell_val = nullptr; d.ell_col = nullptr; d.ell_w = 0;
  rr_status s;
  auto fail = [&](rr_status st) {
    cudaFree(d.coef); cudaFree(d.coef32); cudaFree(d.wsqrt); cudaFree(d.wisqrt); cudaFree(d.flow);
    cudaFree(d.ell_val); cudaFree(d.ell_col);
    delete op;
    return st;
  };
  if ((s = dalloc(&d.coef, N * 9 * q * sizeof(double))) != RR_OK) return fail(s);
  if ((s = dalloc(&d.coef32, N * 9 * q * sizeof(float))) != RR_OK) return fail(s);
  if ((s = dalloc(&d.flow, 3 * npts * sizeof(double))) != RR_OK) return fail(s);
  std::vector<double> hf(3 * npts, 1.0);
  if (fl->rho) std::memcpy(hf.data(), fl->rho, npts * sizeof(double));
  std::memcpy(hf.data() + npts, fl->u, npts * sizeof(double));
  std::memcpy(hf.data() + 2 * npts, fl->v, npts * sizeof(double));
  if (ns)
    for (size_t p = 0; p < npts; ++p)
      if (!(hf[p] > 0.0)) return fail(arg_error("rr_create_operator: rho must be positive"));
  cudaError_t e = cudaMemcpy(d.flow, hf.data(), hf.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMemcpy flow"));
  if (weights) {
    std::vector<double> ws(N), wi(N);
    for (size_t n = 0; n < N; ++n) {
      ws[n] = std::sqrt(weights[n]);
      wi[n] = 1.0 / ws[n];
    }
    if ((s = dalloc(&d.wsqrt, N * sizeof(double))) != RR_OK) return fail(s);
    if ((s = dalloc(&d.wisqrt, N * sizeof(double))) != RR_OK) return fail(s);
    e = cudaMemcpy(d.wsqrt, ws.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.wisqrt, wi.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaMemcpy weights"));
  }
  if ((s = launch_assemble(d, *g, 0)) != RR_OK) return fail(s);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_status(e, "operator assembly"));
  if ((s = build_ell(d)) != RR_OK) return fail(s);
  *out = op;
  return RR_OK;
}

extern "C" rr_status rr_destroy_operator(rr_operator* op) {
  if (!op) return RR_OK;
  DeviceGuard guard(op->d.device);
  cudaFree(op->d.coef);
  cudaFree(op->d.coef32);
  cudaFree(op->d.ell_val);
  cudaFree(op->d.ell_col);
  cudaFree(op->d.wsqrt);
  cudaFree(op->d.wisqrt);
  cudaFree(op->d.flow);
  delete op;
  return RR_OK;
}

extern "C" rr_status rr_operator_dims(const rr_operator* op, int* n, int* b, int* q, int* nx,
                                      int* ny) {
  if (!op) return arg_error("rr_operator_dims: null operator");
  if (n) *n = op->d.n;
  if (b) *b = op->d.b;
  if (q) *q = op->d.q;
  if (nx) *nx = op->d.nx;
  if (ny) *ny = op->d.ny;
  return RR_OK;
}

extern "C" rr_status rr_apply(rr_operator* op, int nshift, const double* shifts, int k, int adjoint,
                              const void* x, void* y, void* stream) {
  if (!op || !shifts || !x || !y) return arg_error("rr_apply: null argument");
  if (nshift < 1 || k < 1) return arg_error("rr_apply: nshift and k must be >= 1");
  if (x == y) return arg_error("rr_apply: x and y must be distinct");
  DeviceGuard guard(op->d.device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double2* sd = nullptr;
  rr_status s = dalloc(&sd, nshift * sizeof(double2));
  if (s != RR_OK) return s;
  cudaError_t e = cudaMemcpyAsync(sd, shifts, nshift * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { cudaFree(sd); return cuda_status(e, "rr_apply shifts"); }
  // bi-global operators: y = D (s I - L~) D^{-1} x with the real L~ = D^{-1} L D
  // (the adjoint likewise, D unitary); D^{-1} x goes through a temporary
  double2* xt = nullptr;
  const double2* xin = (const double2*)x;
  if (op->d.q == 4) {
    const size_t bytes = (size_t)nshift * op->d.n * k * sizeof(double2);
    s = dalloc(&xt, bytes);
    if (s == RR_OK) e = cudaMemcpyAsync(xt, x, bytes, cudaMemcpyDeviceToDevice, st);
    if (s == RR_OK && e == cudaSuccess) s = launch_kz_phase(nshift, op->d.n, k, 4, -1, xt, st);
    if (s != RR_OK || e != cudaSuccess) {
      cudaFree(sd);
      cudaFree(xt);
      return s != RR_OK ? s : cuda_status(e, "rr_apply");
    }
    xin = xt;
  }
  s = launch_apply(op->d, nshift, sd, k, adjoint, xin, (double2*)y, st);
  if (s == RR_OK) s = launch_kz_phase(nshift, op->d.n, k, op->d.q, 1, (double2*)y, st);
  e = cudaStreamSynchronize(st);
  cudaFree(sd);
  cudaFree(xt);
  if (s != RR_OK) return s;
  if (e != cudaSuccess) return cuda_status(e, "rr_apply");
  return RR_OK;
}

extern "C" rr_status rr_phi(rr_operator* op, double* phi, void* stream) {
  if (!op || !phi) return arg_error("rr_phi: null argument");
  DeviceGuard guard(op->d.device);
  return launch_phi(op->d, phi, reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------------ factors
extern "C" rr_status rr_factor(rr_operator* op, int nshift, const double* shifts, rr_precision prec,
                               void* stream, rr_factors** out) {
  if (!op || !shifts || !out) return arg_error("rr_factor: null argument");
  *out = nullptr;
  if (nshift < 1 || nshift > 65535) return arg_error("rr_factor: nshift must be in [1, 65535]");
  if (prec != RR_FP64 && prec != RR_FP32 && prec != RR_FP32_SIMT && prec != RR_FP32_BF16X3 &&
      prec != RR_FP32_BF16X6)
    return arg_error("rr_factor: unknown precision");
  for (int f = 0; f < 2 * nshift; ++f)
    if (!std::isfinite(shifts[f])) return arg_error("rr_factor: shifts must be finite");
  DeviceGuard guard(op->d.device);
  const OpDev& d = op->d;
  rr_factors* fa = new rr_factors();
  std::memset(fa, 0, sizeof(*fa));
  fa->op = op;
  fa->F = nshift;
  fa->prec = prec;
  fa->stream = reinterpret_cast<cudaStream_t>(stream);
  fa->csz = prec == RR_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t bb = (size_t)d.b * d.b;
  rr_status s;
  auto fail = [&](rr_status st) {
    rr_destroy_factors(fa);
    return st;
  };
  if ((s = dalloc(&fa->G, (size_t)nshift * d.nx * bb * fa->csz)) != RR_OK) return fail(s);
  if ((s = dalloc(&fa->X, (size_t)nshift * bb * fa->csz)) != RR_OK) return fail(s);
  if ((s = dalloc(&fa->M, (size_t)nshift * bb * fa->csz)) != RR_OK) return fail(s);
  if ((s = dalloc(&fa->Bbuf, (size_t)nshift * 32 * d.b * fa->csz)) != RR_OK) return fail(s);
  if ((s = dalloc(&fa->Tbuf, (size_t)nshift * 128 * d.b * fa->csz)) != RR_OK) return fail(s);
  if (tc_prec(prec)) {
    if ((s = dalloc(&fa->Pbuf, (size_t)4 * nshift * 64 * d.b * sizeof(float2))) != RR_OK)
      return fail(s);
    fa->tma_ok = encode_factor_maps(fa);
    fa->tma_m_ok = encode_m_map(fa);
    if (d.b >= 64 && d.b <= 768 && d.b % 8 == 0) {
      if ((s = dalloc(&fa->rowpiv, (size_t)nshift * d.b * sizeof(int))) != RR_OK) return fail(s);
      if ((s = dalloc(&fa->pivslot, (size_t)nshift * d.b * sizeof(int))) != RR_OK) return fail(s);
      if ((s = dalloc(&fa->Wbuf, (size_t)nshift * 128 * d.b * sizeof(float2))) != RR_OK)
        return fail(s);
      fa->wide_ok = encode_wide_maps(fa);
    }
  }
  if ((s = dalloc(&fa->perm, (size_t)nshift * d.b * sizeof(int))) != RR_OK) return fail(s);
  if ((s = dalloc(&fa->ipiv, (size_t)nshift * 32 * sizeof(int))) != RR_OK) return fail(s);
  // flags: one singular-pivot flag per shift, then the tensor-core wait flag,
  // then room for the active-problem list of the refinement
  if ((s = dalloc(&fa->flag, (size_t)(2 * nshift + 1) * sizeof(int))) != RR_OK) return fail(s);
  fa->amap_buf = fa->flag + nshift + 1;
  if ((s = dalloc(&fa->shifts, (size_t)nshift * sizeof(double2))) != RR_OK) return fail(s);
  {
    // the look-ahead panel stream gets the highest priority so its CTAs are
    // scheduled ahead of the trailing update's as SMs free up
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    cudaError_t e1 = cudaStreamCreateWithPriority(&fa->stream2, cudaStreamNonBlocking, hi_prio);
    if (e1 == cudaSuccess)
      e1 = cudaStreamCreateWithPriority(&fa->stream3, cudaStreamNonBlocking, hi_prio);
    if (e1 == cudaSuccess) e1 = cudaEventCreateWithFlags(&fa->ev_next, cudaEventDisableTiming);
    if (e1 == cudaSuccess) e1 = cudaEventCreateWithFlags(&fa->ev_panel, cudaEventDisableTiming);
    for (int q = 0; q < 9 && e1 == cudaSuccess; ++q)
      e1 = cudaEventCreateWithFlags(&fa->ev_w[q], cudaEventDisableTiming);
    if (e1 != cudaSuccess) return fail(cuda_status(e1, "rr_factor: stream/event creation"));
  }
  fa->shifts_h = new double2[nshift];
  for (int f = 0; f < nshift; ++f) fa->shifts_h[f] = make_double2(shifts[2 * f], shifts[2 * f + 1]);
  cudaStream_t st = fa->stream;
  cudaError_t e = cudaMemcpyAsync(fa->shifts, fa->shifts_h, nshift * sizeof(double2),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(cuda_status(e, "rr_factor shifts"));
  e = cudaMemsetAsync(fa->flag, 0, (nshift + 1) * sizeof(int), st);
  if (e != cudaSuccess) return fail(cuda_status(e, "rr_factor flags"));
  if ((s = launch_factor(fa)) != RR_OK) return fail(s);
  std::vector<int> flags(nshift + 1);
  e = cudaMemcpyAsync(flags.data(), fa->flag, (nshift + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                      st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_status(e, "rr_factor"));
  if (flags[nshift]) {
    g_err = "rr_factor: a tensor-core update kernel timed out waiting for its MMAs";
    return fail(RR_ERR_TIMEOUT);
  }
  *out = fa;
  for (int f = 0; f < nshift; ++f)
    if (flags[f]) {
      char buf[128];
      snprintf(buf, sizeof buf, "rr_factor: exact zero pivot for shift %d (%g%+gi)", f,
               fa->shifts_h[f].x, fa->shifts_h[f].y);
      g_err = buf;
      return RR_ERR_SINGULAR;
    }
  return RR_OK;
}

extern "C" rr_status rr_destroy_factors(rr_factors* fa) {
  if (!fa) return RR_OK;
  DeviceGuard guard(fa->op->d.device);
  if (fa->stream) cudaStreamSynchronize(fa->stream);
  if (!fa->is_view) {
    cudaFree(fa->G);
    cudaFree(fa->shifts);
  }
  cudaFree(fa->chk);
  delete fa->sched;
  delete fa->chk_desc;
  cudaFree(fa->X);
  cudaFree(fa->M);
  cudaFree(fa->Bbuf);
  cudaFree(fa->Tbuf);
  cudaFree(fa->Pbuf);
  cudaFree(fa->perm);
  cudaFree(fa->ipiv);
  cudaFree(fa->rowpiv);
  cudaFree(fa->pivslot);
  cudaFree(fa->Wbuf);
  cudaFree(fa->flag);
  cudaFree(fa->ws);
  if (fa->stream2) {
    cudaStreamSynchronize(fa->stream2);
    cudaStreamDestroy(fa->stream2);
  }
  if (fa->stream3) {
    cudaStreamSynchronize(fa->stream3);
    cudaStreamDestroy(fa->stream3);
  }
  if (fa->ev_next) cudaEventDestroy(fa->ev_next);
  if (fa->ev_panel) cudaEventDestroy(fa->ev_panel);
  for (int q = 0; q < 9; ++q)
    if (fa->ev_w[q]) cudaEventDestroy(fa->ev_w[q]);
  delete[] fa->shifts_h;
  delete fa;
  return RR_OK;
}

// ------------------------------------------------ batch-plan internals
// View over shifts [f0, f0 + nf) of parent factors: shares G and the device
// shifts, owns staging buffers, flags, workspace and TMA maps.
rr_status factors_view(rr_factors* parent, int f0, int nf, cudaStream_t st, rr_factors** out) {
  *out = nullptr;
  if (!parent || parent->is_view || f0 < 0 || nf < 1 || f0 + nf > parent->F)
    return arg_error("factors_view: bad range");
  DeviceGuard guard(parent->op->d.device);
  const OpDev& d = parent->op->d;
  rr_factors* v = new rr_factors();
  std::memset(v, 0, sizeof(*v));
  v->op = parent->op;
  v->F = nf;
  v->prec = parent->prec;
  v->stream = st;
  v->csz = parent->csz;
  v->is_view = 1;
  v->G = static_cast<char*>(parent->G) + (size_t)f0 * d.nx * d.b * d.b * parent->csz;
  v->shifts = parent->shifts + f0;
  v->tune_update = parent->tune_update;
  rr_status s;
  auto fail = [&](rr_status r) {
    rr_destroy_factors(v);
    return r;
  };
  if ((s = dalloc(&v->Tbuf, (size_t)nf * 128 * d.b * v->csz)) != RR_OK) return fail(s);
  if (tc_prec(v->prec)) {
    if ((s = dalloc(&v->Pbuf, (size_t)4 * nf * 64 * d.b * sizeof(float2))) != RR_OK) return fail(s);
    v->tma_ok = encode_factor_maps(v);
  }
  if ((s = dalloc(&v->flag, (size_t)(2 * nf + 1) * sizeof(int))) != RR_OK) return fail(s);
  v->amap_buf = v->flag + nf + 1;
  RR_CUDA(cudaMemsetAsync(v->flag, 0, (nf + 1) * sizeof(int), st));
  v->shifts_h = new double2[nf];
  for (int f = 0; f < nf; ++f) v->shifts_h[f] = parent->shifts_h[f0 + f];
  v->sched = new std::vector<int>();
  v->chk_desc = new std::vector<long long>();
  *out = v;
  return RR_OK;
}

// Factorisation launches only (flags cleared first, no host synchronisation):
// the form a graph captures.  Flags are read by factor_flags afterwards.
rr_status factor_async(rr_factors* fa) {
  if (fa->is_view) return arg_error("factor_async: a view cannot be factored");
  DeviceGuard guard(fa->op->d.device);
  RR_CUDA(cudaMemsetAsync(fa->flag, 0, (fa->F + 1) * sizeof(int), fa->stream));
  return launch_factor(fa);
}

rr_status factor_flags(rr_factors* fa) {
  DeviceGuard guard(fa->op->d.device);
  std::vector<int> flags(fa->F + 1);
  RR_CUDA(cudaMemcpy(flags.data(), fa->flag, (fa->F + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (flags[fa->F]) {
    g_err = "a tensor-core update kernel timed out waiting for its MMAs";
    return RR_ERR_TIMEOUT;
  }
  for (int f = 0; f < fa->F; ++f)
    if (flags[f]) {
      g_err = "exact zero pivot in a batched factorisation";
      return RR_ERR_SINGULAR;
    }
  return RR_OK;
}

// Workspace for k columns allocated ahead of a capture (no allocation may
// happen while a graph is recorded).
rr_status factors_reserve(rr_factors* fa, int k) {
  DeviceGuard guard(fa->op->d.device);
  Work w;
  return get_work(fa, k, &w);
}

// Milliseconds of one unrefined forward solve with k columns on zeroed
// inputs (autotuner timing of the sweep schedule); the first run warms up.
rr_status time_solve(rr_factors* fa, int k, float* ms) {
  DeviceGuard guard(fa->op->d.device);
  Work w;
  rr_status s = get_work(fa, k, &w);
  if (s != RR_OK) return s;
  cudaStream_t st = fa->stream;
  const size_t nel = (size_t)fa->F * fa->op->d.n * k;
  RR_CUDA(cudaMemsetAsync(w.L1, 0, nel * fa->csz, st));
  cudaEvent_t e0, e1;
  RR_CUDA(cudaEventCreate(&e0));
  RR_CUDA(cudaEventCreate(&e1));
  s = launch_solve_lo(fa, k, 0, w.L1, w.L2, w.L3);
  if (s == RR_OK) {
    cudaEventRecord(e0, st);
    s = launch_solve_lo(fa, k, 0, w.L1, w.L2, w.L3);
    cudaEventRecord(e1, st);
  }
  cudaError_t e = cudaEventSynchronize(e1);
  if (s == RR_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != RR_OK) return s;
  if (e != cudaSuccess) return cuda_status(e, "time_solve");
  return RR_OK;
}

extern "C" rr_status rr_factors_dims(const rr_factors* fa, int* nshift, int* prec) {
  if (!fa) return arg_error("rr_factors_dims: null factors");
  if (nshift) *nshift = fa->F;
  if (prec) *prec = fa->prec;
  return RR_OK;
}

static rr_status check_k(rr_factors* fa, int k, const char* who) {
  if (!fa) return arg_error(std::string(who) + ": null factors");
  if (k < 1 || k > 64) return arg_error(std::string(who) + ": k must be in [1, 64]");
  if (k > fa->op->d.n) return arg_error(std::string(who) + ": k must not exceed N");
  return RR_OK;
}

extern "C" rr_status rr_solve(rr_factors* fa, int k, int adjoint, const void* b, void* x,
                              double refine_tol, int max_refine, rr_info* info) {
  rr_status s = check_k(fa, k, "rr_solve");
  if (s != RR_OK) return s;
  if (!b || !x) return arg_error("rr_solve: null vector");
  if (b == x) return arg_error("rr_solve: b and x must be distinct");
  if (max_refine < 0) return arg_error("rr_solve: max_refine must be >= 0");
  DeviceGuard guard(fa->op->d.device);
  info_reset(info);
  Work w;
  if ((s = get_work(fa, k, &w)) != RR_OK) return s;
  const OpDev& d = fa->op->d;
  const int F = fa->F;
  const size_t bytes = (size_t)F * d.n * k * sizeof(double2);
  cudaStream_t st = fa->stream;
  // R b = W^{1/2} A^{-1} W^{-1/2} b ;  R^H b = W^{-1/2} A^{-H} W^{1/2} b
  // (bi-global operators: the solve runs on D^{-1} L D, D = diag(1, 1, 1, i))
  RR_CUDA(cudaMemcpyAsync(w.W2, b, bytes, cudaMemcpyDeviceToDevice, st));
  if ((s = launch_kz_phase(F, d.n, k, d.q, -1, w.W2, st)) != RR_OK) return s;
  if ((s = launch_scale_rows(F, d.n, k, adjoint ? d.wsqrt : d.wisqrt, w.W2, st)) != RR_OK) return s;
  s = solve_refined(fa, k, adjoint, w.W2, (double2*)x, refine_tol, max_refine, w, info);
  if (s != RR_OK && s != RR_ERR_NOCONV) return s;
  rr_status s2 = launch_scale_rows(F, d.n, k, adjoint ? d.wisqrt : d.wsqrt, (double2*)x, st);
  if (s2 == RR_OK) s2 = launch_kz_phase(F, d.n, k, d.q, 1, (double2*)x, st);
  if (s2 != RR_OK) return s2;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "rr_solve");
  return s;
}

static rr_status check_opts(const rr_sketch_opts* o, const char* who) {
  if (!o) return RR_OK;
  if (o->omega_kind < RR_OMEGA_GAUSSIAN || o->omega_kind > RR_OMEGA_ORTHONORMAL)
    return arg_error(std::string(who) + ": unknown omega_kind");
  if (o->omega_kind == RR_OMEGA_SPARSE_RADEMACHER && !(o->density > 0.0 && o->density <= 1.0))
    return arg_error(std::string(who) + ": density must be in (0, 1]");
  if (o->power_iters < 0 || o->power_iters > 64)
    return arg_error(std::string(who) + ": power_iters must be in [0, 64]");
  return RR_OK;
}

extern "C" rr_status rr_sketch_ex(rr_factors* fa, int k, const uint64_t* seeds, const double* phi,
                                  const rr_sketch_opts* opts, double refine_tol, int max_refine,
                                  void* V, double* sigma_halko, rr_info* info) {
  rr_status s = check_k(fa, k, "rr_sketch");
  if (s != RR_OK) return s;
  if (!seeds || !V || !sigma_halko) return arg_error("rr_sketch: null argument");
  if (max_refine < 0) return arg_error("rr_sketch: max_refine must be >= 0");
  if ((s = check_opts(opts, "rr_sketch")) != RR_OK) return s;
  const int kind = opts ? opts->omega_kind : RR_OMEGA_GAUSSIAN;
  const int power_iters = opts ? opts->power_iters : 0;
  DeviceGuard guard(fa->op->d.device);
  info_reset(info);
  Work w;
  if ((s = get_work(fa, k, &w)) != RR_OK) return s;
  const OpDev& d = fa->op->d;
  const int F = fa->F, N = d.n;
  const size_t bytes = (size_t)F * N * k * sizeof(double2);
  cudaStream_t st = fa->stream;
  rr_status conv = RR_OK;
  auto note = [&](rr_status r) {
    if (r == RR_ERR_NOCONV) conv = r;
    return r == RR_ERR_NOCONV ? RR_OK : r;
  };
  // (replayed launch sequences reuse the seeds the recording run uploaded)
  if (fa->sched_mode != SCHED_REPLAY)
    RR_CUDA(cudaMemcpyAsync(w.seeds, seeds, F * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  // Omega' = W^{-1/2} diag(phi) Omega  (first step, Eq. 9)
  if (kind == RR_OMEGA_ORTHONORMAL) {
    // Omega = Q factor of diag(phi) randn (CholeskyQR2), then weighted
    if ((s = launch_philox(F, N, k, w.seeds, phi, nullptr, w.W1, st, 0)) != RR_OK) return s;
    if ((s = cholqr2(fa, k, w.W1, nullptr, w, info)) != RR_OK) return s;
    if ((s = launch_scale_rows(F, N, k, d.wisqrt, w.W1, st)) != RR_OK) return s;
  } else {
    const double dens = opts ? opts->density : 1.0;
    if ((s = launch_philox(F, N, k, w.seeds, phi, d.wisqrt, w.W1, st, kind, dens)) != RR_OK)
      return s;
  }
  // (bi-global operators: everything below runs on D^{-1} L D, so Omega
  // enters as D^{-1} Omega and V leaves as D V)
  if ((s = launch_kz_phase(F, N, k, d.q, -1, w.W1, st)) != RR_OK) return s;
  // Y = W^{1/2} A^{-1} Omega'  (second step)
  if ((s = note(solve_refined(fa, k, 0, w.W1, w.W2, refine_tol, max_refine, w, info))) != RR_OK)
    return s;
  if ((s = launch_scale_rows(F, N, k, d.wsqrt, w.W2, st)) != RR_OK) return s;
  // Q = qr(Y)  (third step)
  if ((s = cholqr2(fa, k, w.W2, nullptr, w, info)) != RR_OK) return s;
  // subspace iterations: Z = qr(R^H Q), Q = qr(R Z)
  for (int it = 0; it < power_iters; ++it) {
    RR_CUDA(cudaMemcpyAsync(w.W1, w.W2, bytes, cudaMemcpyDeviceToDevice, st));
    if ((s = launch_scale_rows(F, N, k, d.wsqrt, w.W1, st)) != RR_OK) return s;
    if ((s = note(solve_refined(fa, k, 1, w.W1, w.W3, refine_tol, max_refine, w, info))) != RR_OK)
      return s;
    if ((s = launch_scale_rows(F, N, k, d.wisqrt, w.W3, st)) != RR_OK) return s;
    if ((s = cholqr2(fa, k, w.W3, nullptr, w, info)) != RR_OK) return s;
    RR_CUDA(cudaMemcpyAsync(w.W1, w.W3, bytes, cudaMemcpyDeviceToDevice, st));
    if ((s = launch_scale_rows(F, N, k, d.wisqrt, w.W1, st)) != RR_OK) return s;
    if ((s = note(solve_refined(fa, k, 0, w.W1, w.W2, refine_tol, max_refine, w, info))) != RR_OK)
      return s;
    if ((s = launch_scale_rows(F, N, k, d.wsqrt, w.W2, st)) != RR_OK) return s;
    if ((s = cholqr2(fa, k, w.W2, nullptr, w, info)) != RR_OK) return s;
  }
  // B^H = W^{-1/2} A^{-H} W^{1/2} Q  (fourth step)
  RR_CUDA(cudaMemcpyAsync(w.W1, w.W2, bytes, cudaMemcpyDeviceToDevice, st));
  if ((s = launch_scale_rows(F, N, k, d.wsqrt, w.W1, st)) != RR_OK) return s;
  if ((s = note(solve_refined(fa, k, 1, w.W1, w.W3, refine_tol, max_refine, w, info))) != RR_OK)
    return s;
  if ((s = launch_scale_rows(F, N, k, d.wisqrt, w.W3, st)) != RR_OK) return s;
  // svd(B): B^H = Q_B R_B, R_B = Ul S Vr^H  =>  V = Q_B Ul, sigma = S  (fifth step);
  // Q_B = Y1 R_last^{-1} is not formed: V = Y1 (R_last^{-1} Ul)
  if ((s = cholqr2(fa, k, w.W3, w.R2i, w, info, w.Rd)) != RR_OK) return s;
  if ((s = launch_jacobi_svd(F, k, w.R2i, w.sig, w.Ul, w.Vr, w.sweeps, st)) != RR_OK) return s;
  if ((s = launch_small_mul(F, k, w.Rd, w.Ul, w.R1, st)) != RR_OK) return s;
  if ((s = launch_right_mul(F, N, k, w.W3, w.R1, (double2*)V, st)) != RR_OK) return s;
  if ((s = launch_kz_phase(F, N, k, d.q, 1, (double2*)V, st)) != RR_OK) return s;
  RR_CUDA(cudaMemcpyAsync(sigma_halko, w.sig, (size_t)F * k * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (fa->sched_mode != SCHED_REPLAY) RR_CUDA(cudaStreamSynchronize(st));
  return conv;
}

extern "C" rr_status rr_sketch(rr_factors* fa, int k, const uint64_t* seeds, const double* phi,
                               double refine_tol, int max_refine, void* V, double* sigma_halko,
                               rr_info* info) {
  return rr_sketch_ex(fa, k, seeds, phi, nullptr, refine_tol, max_refine, V, sigma_halko, info);
}

extern "C" rr_status rr_modes(rr_factors* fa, int k, void* V, void* U, double* sigma,
                              int orthogonalize, double refine_tol, int max_refine, rr_info* info) {
  rr_status s = check_k(fa, k, "rr_modes");
  if (s != RR_OK) return s;
  if (!V || !U || !sigma) return arg_error("rr_modes: null argument");
  if (U == V) return arg_error("rr_modes: U and V must be distinct");
  if (max_refine < 0) return arg_error("rr_modes: max_refine must be >= 0");
  DeviceGuard guard(fa->op->d.device);
  info_reset(info);
  Work w;
  if ((s = get_work(fa, k, &w)) != RR_OK) return s;
  const OpDev& d = fa->op->d;
  const int F = fa->F, N = d.n;
  const size_t bytes = (size_t)F * N * k * sizeof(double2);
  cudaStream_t st = fa->stream;
  rr_status conv = RR_OK;
  // U Sigma = W^{1/2} A^{-1} W^{-1/2} V  (Eq. 8)
  // (bi-global operators: the solve runs on D^{-1} L D, D = diag(1, 1, 1, i))
  RR_CUDA(cudaMemcpyAsync(w.W1, V, bytes, cudaMemcpyDeviceToDevice, st));
  if ((s = launch_kz_phase(F, N, k, d.q, -1, w.W1, st)) != RR_OK) return s;
  if ((s = launch_scale_rows(F, N, k, d.wisqrt, w.W1, st)) != RR_OK) return s;
  s = solve_refined(fa, k, 0, w.W1, w.W2, refine_tol, max_refine, w, info);
  if (s == RR_ERR_NOCONV) conv = s; else if (s != RR_OK) return s;
  if ((s = launch_scale_rows(F, N, k, d.wsqrt, w.W2, st)) != RR_OK) return s;
  if ((s = launch_kz_phase(F, N, k, d.q, 1, w.W2, st)) != RR_OK) return s;
  if (!orthogonalize) {
    // sigma_j = ||(U Sigma)_j||, u_j = (U Sigma)_j / sigma_j
    if ((s = launch_colnorm2(F, N, k, w.W2, w.dpart, w.nblk_col, sigma, st)) != RR_OK) return s;
    if ((s = launch_col_scale(F, N, k, w.W2, sigma, (double2*)U, st)) != RR_OK) return s;
  } else {
    // optional: svd(U Sigma) = U S Vt^H via CholeskyQR2 + Jacobi; V <- V Vt
    if ((s = cholqr2(fa, k, w.W2, w.R2i, w, info, w.Rd)) != RR_OK) return s;
    if ((s = launch_jacobi_svd(F, k, w.R2i, sigma, w.Ul, w.Vr, w.sweeps, st)) != RR_OK) return s;
    if ((s = launch_small_mul(F, k, w.Rd, w.Ul, w.R1, st)) != RR_OK) return s;
    if ((s = launch_right_mul(F, N, k, w.W2, w.R1, (double2*)U, st)) != RR_OK) return s;
    if ((s = launch_right_mul(F, N, k, (const double2*)V, w.Vr, (double2*)V, st)) != RR_OK) return s;
  }
  if ((s = launch_finish_modes(F, N, k, (double2*)U, (double2*)V, sigma, w.W1, w.W3, w.dpart,
                               w.nblk_col, w.rank, w.phase, st)) != RR_OK)
    return s;
  if (fa->sched_mode != SCHED_REPLAY) RR_CUDA(cudaStreamSynchronize(st));
  return conv;
}

extern "C" rr_status rr_gain_grad(rr_factors* fa, int k, int J, const void* U, const void* V,
                                  const double* sigma, double refine_tol, int max_refine,
                                  double* grad, rr_info* info) {
  rr_status s = check_k(fa, k, "rr_gain_grad");
  if (s != RR_OK) return s;
  if (!U || !V || !sigma || !grad) return arg_error("rr_gain_grad: null argument");
  if (J < 1 || J > k) return arg_error("rr_gain_grad: J must be in [1, k]");
  if (max_refine < 0) return arg_error("rr_gain_grad: max_refine must be >= 0");
  if (fa->op->d.q == 4) {
    g_err = "rr_gain_grad: not implemented for the bi-global operator";
    return RR_ERR_UNSUPPORTED;
  }
  DeviceGuard guard(fa->op->d.device);
  info_reset(info);
  Work w;
  if ((s = get_work(fa, J, &w)) != RR_OK) return s;
  const OpDev& d = fa->op->d;
  const int F = fa->F, N = d.n;
  cudaStream_t st = fa->stream;
  rr_status conv = RR_OK;
  // first J columns of U and V: [F][N][k] -> [F][N][J]
  const size_t rows = (size_t)F * N;
  // a_j = A^{-H} W^{1/2} u_j
  RR_CUDA(cudaMemcpy2DAsync(w.W1, J * sizeof(double2), U, k * sizeof(double2),
                            J * sizeof(double2), rows, cudaMemcpyDeviceToDevice, st));
  if ((s = launch_scale_rows(F, N, J, d.wsqrt, w.W1, st)) != RR_OK) return s;
  s = solve_refined(fa, J, 1, w.W1, w.W2, refine_tol, max_refine, w, info);
  if (s == RR_ERR_NOCONV) conv = s; else if (s != RR_OK) return s;
  // b_j = A^{-1} W^{-1/2} v_j
  RR_CUDA(cudaMemcpy2DAsync(w.W1, J * sizeof(double2), V, k * sizeof(double2),
                            J * sizeof(double2), rows, cudaMemcpyDeviceToDevice, st));
  if ((s = launch_scale_rows(F, N, J, d.wisqrt, w.W1, st)) != RR_OK) return s;
  s = solve_refined(fa, J, 0, w.W1, w.W3, refine_tol, max_refine, w, info);
  if (s == RR_ERR_NOCONV) conv = s; else if (s != RR_OK) return s;
  if ((s = launch_gain_grad(d, fa->op->grid, F, J, w.W2, w.W3, sigma, k, w.featbar, grad, st)) !=
      RR_OK)
    return s;
  RR_CUDA(cudaStreamSynchronize(st));
  return conv;
}

extern "C" rr_status rr_refactor(rr_factors* fa, const double* shifts) {
  if (!fa || !shifts) return arg_error("rr_refactor: null argument");
  if (fa->is_view) return arg_error("rr_refactor: factors owned by a batch plan");
  const int F = fa->F;
  for (int f = 0; f < 2 * F; ++f)
    if (!std::isfinite(shifts[f])) return arg_error("rr_refactor: shifts must be finite");
  DeviceGuard guard(fa->op->d.device);
  cudaStream_t st = fa->stream;
  // the previous work on the stream may still read shifts_h-derived data
  RR_CUDA(cudaStreamSynchronize(st));
  for (int f = 0; f < F; ++f) fa->shifts_h[f] = make_double2(shifts[2 * f], shifts[2 * f + 1]);
  RR_CUDA(cudaMemcpyAsync(fa->shifts, fa->shifts_h, F * sizeof(double2), cudaMemcpyHostToDevice, st));
  RR_CUDA(cudaMemsetAsync(fa->flag, 0, (F + 1) * sizeof(int), st));
  rr_status s = launch_factor(fa);
  if (s != RR_OK) return s;
  std::vector<int> flags(F + 1);
  RR_CUDA(cudaMemcpyAsync(flags.data(), fa->flag, (F + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  if (flags[F]) {
    g_err = "rr_refactor: a tensor-core update kernel timed out waiting for its MMAs";
    return RR_ERR_TIMEOUT;
  }
  for (int f = 0; f < F; ++f)
    if (flags[f]) {
      g_err = "rr_refactor: exact zero pivot";
      return RR_ERR_SINGULAR;
    }
  return RR_OK;
}

extern "C" rr_status rr_gaussian(int nshift, int n, int k, const uint64_t* seeds, const double* phi,
                                 void* omega, void* stream) {
  return rr_test_matrix(nshift, n, k, seeds, phi, RR_OMEGA_GAUSSIAN, 1.0, omega, stream);
}

extern "C" rr_status rr_test_matrix(int nshift, int n, int k, const uint64_t* seeds,
                                    const double* phi, int kind, double density, void* omega,
                                    void* stream) {
  if (!seeds || !omega) return arg_error("rr_test_matrix: null argument");
  if (nshift < 1 || n < 1 || k < 1) return arg_error("rr_test_matrix: sizes must be >= 1");
  if (kind < RR_OMEGA_GAUSSIAN || kind > RR_OMEGA_SPARSE_RADEMACHER)
    return arg_error("rr_test_matrix: kind must be Gaussian, Rademacher or sparse Rademacher");
  if (kind == RR_OMEGA_SPARSE_RADEMACHER && !(density > 0.0 && density <= 1.0))
    return arg_error("rr_test_matrix: density must be in (0, 1]");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* sd = nullptr;
  rr_status s = dalloc(&sd, nshift * sizeof(uint64_t));
  if (s != RR_OK) return s;
  cudaError_t e = cudaMemcpyAsync(sd, seeds, nshift * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    s = launch_philox(nshift, n, k, sd, phi, nullptr, (double2*)omega, st, kind, density);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(sd);
  if (e != cudaSuccess) return cuda_status(e, "rr_test_matrix");
  return s;
}
