// Internal declarations shared by the CUDA translation units of librr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rr.h"

// ------------------------------------------------------------ complex math
// Interleaved complex in the CUDA vector types: .x = re, .y = im.
template <typename T> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename T> using C_t = typename cplx_t<T>::type;

__host__ __device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 mk(float r, float i) { return make_float2(r, i); }
template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cneg(C a) { return mk(-a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c + a*b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c + conj(a)*b
template <typename C> __device__ __forceinline__ C cfmac(C a, C b, C c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
// c + r*b (r real)
template <typename C, typename R> __device__ __forceinline__ C crfma(R r, C b, C c) {
  c.x = fma(r, b.x, c.x);
  c.y = fma(r, b.y, c.y);
  return c;
}
template <typename C> __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }
template <typename C> __device__ __forceinline__ C cinv(C a) {
  auto d = a.x * a.x + a.y * a.y;
  return mk(a.x / d, -a.y / d);
}
template <typename To, typename From> __device__ __forceinline__ To ccast(From a);
template <> __device__ __forceinline__ double2 ccast<double2, double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 ccast<float2, float2>(float2 a) { return a; }
template <> __device__ __forceinline__ float2 ccast<float2, double2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}
template <> __device__ __forceinline__ double2 ccast<double2, float2>(float2 a) {
  return make_double2((double)a.x, (double)a.y);
}

// ---------------------------------------------------------- operator data
// Stencil of L: for every unknown row n, S = 9*q real coefficients
// coef[n*S + ((dx+1)*3 + (dy+1))*q + c'] = L[n, ((ix+dx)*ny + iy+dy)*q + c'],
// zero where the neighbour is a Dirichlet ghost node.
struct OpDev {
  int kind, q, nx, ny, b, n, periodic;
  double* coef;      // [N][9q]
  float* coef32;     // [N][9q] the same coefficients rounded once to FP32 (FP32 factors)
  // the nonzero stencil entries of every row in stencil order, padded with
  // zero entries on the row itself to a width the FP64 apply kernel is
  // compiled for (ELL layout)
  double* ell_val;   // [N][ell_w]
  int* ell_col;      // [N][ell_w] unknown index of the entry
  int ell_w;
  double* wsqrt;     // [N] W^{1/2} or nullptr (identity)
  double* wisqrt;    // [N] W^{-1/2} or nullptr
  double* flow;      // [3][nx*ny] rho, U, V
  double dx, dy;
  int device;
};

struct rr_operator {
  OpDev d;
  rr_grid grid;
};

// Device-side view of the operator passed by value to kernels.
struct OpView {
  const double* coef;
  const float* coef32;
  const double* ell_val;
  const int* ell_col;
  int q, nx, ny, b, n, periodic, S, ell_w;
};

inline OpView view(const OpDev& d) {
  OpView v;
  v.coef = d.coef;
  v.coef32 = d.coef32;
  v.ell_val = d.ell_val;
  v.ell_col = d.ell_col;
  v.ell_w = d.ell_w;
  v.q = d.q; v.nx = d.nx; v.ny = d.ny; v.b = d.b; v.n = d.n;
  v.periodic = d.periodic; v.S = 9 * d.q;
  return v;
}

// Stencil coefficient in the arithmetic of T: FP64 kernels read the FP64
// array, FP32 kernels its copy rounded once at assembly (the same value a
// conversion at every use would give).
template <typename T> __device__ __forceinline__ T coefv(const OpView& op, size_t idx);
template <> __device__ __forceinline__ double coefv<double>(const OpView& op, size_t idx) {
  return op.coef[idx];
}
template <> __device__ __forceinline__ float coefv<float>(const OpView& op, size_t idx) {
  return op.coef32[idx];
}

// y index of a neighbour; returns -1 for a Dirichlet ghost.
__device__ __forceinline__ int nbr_y(int iy, int dy, int ny, int periodic) {
  int j = iy + dy;
  if (periodic) return (j + ny) % ny;
  return (j < 0 || j >= ny) ? -1 : j;
}

// ------------------------------------------------------------- factors
struct rr_factors {
  rr_operator* op;
  int F;
  int prec;          // rr_precision
  cudaStream_t stream;
  cudaStream_t stream2;  // look-ahead panel stream (owned)
  cudaStream_t stream3;  // slab-update stream of the wide factorisation (owned)
  cudaEvent_t ev_next, ev_panel;
  cudaEvent_t ev_w[9];   // wide factorisation: panel / slab-update rings and the join
  size_t csz;        // bytes of one complex element of the factors
  void* G;           // [F][nx][b][b]   inverse of each Schur block
  void* X;           // [F][b][b] X_i = G_i C_i of the current column (transient)
  void* M;           // [F][b][b] work matrix
  void* Bbuf;        // [F][32][b] saved pivot rows of the current panel
  void* Tbuf;        // [2][F][b][64] staging blocks of one sweep step
  void* Pbuf;        // [4][F][b][64] partial products of the split tensor-core sweep
  alignas(64) unsigned char tmap[3][128];  // TMA maps: G tiles, G^H tiles, M row tiles (FP32)
  int tma_ok;        // 1 if the maps of G were encoded
  int tma_m_ok;      // 1 if the map of M was encoded
  int* perm;         // [F][b]
  int* ipiv;         // [F][32]
  // wide (two-level, implicitly pivoted) factorisation of FP32 factors
  int wide_ok;       // 1 if the buffers and TMA maps below exist
  int* rowpiv;       // [F][b] pivot column of each row (-1: not yet pivoted)
  int* pivslot;      // [F][b] pivot row of each column
  void* Wbuf;        // [F][128][b] gathered pivot rows of a slab (outer update)
  alignas(64) unsigned char wmap[2][128];  // TMA maps: A chunks of M, Wbuf rows
  int* flag;         // [F] singular-pivot flags
  double2* shifts;   // [F] device
  double2* shifts_h; // [F] host copy
  // workspace for the sketch (allocated lazily, sized for kmax)
  int kmax;
  void* ws;          // one allocation, carved below
  size_t ws_bytes;
  // A view (batch plans) aliases the factors G and the device shifts of a
  // parent over a range of its shifts; it owns its staging buffers, flags,
  // workspace and TMA maps, and never runs the factorisation.
  int is_view;
  // Host decisions recorded for graph capture.  SCHED_RECORD runs eagerly and
  // appends every data-dependent decision (refinement corrections per solve,
  // shifted CholeskyQR per QR) to sched; SCHED_REPLAY issues the same launch
  // sequence without host reads, logging residual norms and breakdown flags
  // into the device check log chk for inspection after the graph has run.
  int sched_mode;
  std::vector<int>* sched;      // owned
  size_t sched_pos;
  char* chk;                    // device check log (owned), chk_cap bytes
  size_t chk_cap, chk_off, chk_need;
  std::vector<long long>* chk_desc;  // owned: (kind, byte offset, count) triples
  // tuning overrides (0 = built-in choice): K-split of the tensor-core sweep;
  // 1 = trailing update on the CUDA cores; factor only the first columns
  int tune_ks;
  int tune_update;
  int factor_cols;
  // Active problems of the current refinement correction (eager solves on
  // the tensor-core sweep path): when amap is set, the solve path runs only
  // the Fa problems amap[0..Fa) (device list in amap_buf, which has room for
  // F); otherwise all F.
  int* amap_buf;
  const int* amap;
  int Fa;
  std::vector<int> amap_h;  // host copy of the list
};

// number of problems the solve path runs on, and the problem of slot s
inline int active_count(const rr_factors* fa) { return fa->amap ? fa->Fa : fa->F; }
__device__ __forceinline__ int active_problem(const int* amap, int s) { return amap ? amap[s] : s; }

// Precisions that store complex FP32 factors and run their products on the
// tensor cores (TF32 or BF16 operand splits).
inline bool tc_prec(int prec) {
  return prec == RR_FP32 || prec == RR_FP32_BF16X3 || prec == RR_FP32_BF16X6;
}

enum { SCHED_EAGER = 0, SCHED_RECORD = 1, SCHED_REPLAY = 2 };
enum { CHK_SOLVE = 0, CHK_CQR = 1 };

// ------------------------------------------------------------ error state
void set_error(const std::string& msg);
rr_status cuda_status(cudaError_t e, const char* what);
#define RR_CUDA(call)                                             \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return cuda_status(_e, #call);         \
  } while (0)

// ------------------------------------------------------- kernel launchers
// operator.cu
rr_status launch_assemble(OpDev& d, const rr_grid& g, cudaStream_t st);
// ELL copy of the stencil (allocates ell_val / ell_col; synchronous)
rr_status build_ell(OpDev& d);
rr_status launch_apply(const OpDev& d, int F, const double2* shifts, int k, int adjoint,
                       const double2* x, double2* y, cudaStream_t st);
// r = b - (s I - L) x (or the adjoint); with amap, grid slot f runs problem
// amap[f] (F slots), else problem f
rr_status launch_residual(const OpDev& d, int F, const double2* shifts, int k, int adjoint,
                          const double2* b, const double2* x, double2* r, cudaStream_t st,
                          const int* amap = nullptr);
rr_status launch_phi(const OpDev& d, double* phi, cudaStream_t st);

// rr_api.cu: views over factors and graph-mode helpers of batch plans
rr_status factors_view(rr_factors* parent, int f0, int nf, cudaStream_t st, rr_factors** out);
rr_status factor_async(rr_factors* fa);
rr_status factor_flags(rr_factors* fa);
rr_status factors_reserve(rr_factors* fa, int k);
rr_status time_solve(rr_factors* fa, int k, float* ms);

// factor.cu
rr_status launch_factor(rr_factors* f);
int factor_panel_width(int prec, int b);
// M = D_i - A_i X_{i-1} for FP32 factors (the Schur update of column i)
rr_status launch_schur_f32(rr_factors* f, int i, cudaStream_t st);
// factor_w.cu: the wide FP32 factorisation (TF32 or BF16 operand splits)
bool factor_wide_ok(const rr_factors* f);
rr_status launch_factor_wide(rr_factors* f);

// sweep.cu: x = A^{-1} b or A^{-H} b with the factors in precision T.
// b and x are [F][N][k] in the factor precision; tmp same size (adjoint only).
rr_status launch_solve_lo(rr_factors* f, int k, int adjoint, const void* b, void* x, void* tmp);
// true when the solves of k columns take the split tensor-core sweep, the
// one path that can run on a subset of the problems (rr_factors::amap)
bool sweep_tc2_ok(const rr_factors* f, int k);

// dense.cu
// kind: 0 Gaussian, 1 Rademacher, 2 sparse Rademacher of the given density
rr_status launch_philox(int F, int N, int k, const uint64_t* seeds_dev, const double* phi,
                        const double* wisqrt, double2* out, cudaStream_t st, int kind = 0,
                        double density = 1.0);
rr_status launch_scale_rows(int F, int N, int k, const double* w, double2* x, cudaStream_t st);
// bi-global operators (q = 4): x <- D x (sign > 0) or D^{-1} x, D = diag(1, 1, 1, i)
// per point; no-op for q != 4
rr_status launch_kz_phase(int F, int N, int k, int q, int sign, double2* x, cudaStream_t st);
rr_status launch_convert_d2f(size_t n, const double2* in, float2* out, cudaStream_t st);
rr_status launch_convert_f2d(size_t n, const float2* in, double2* out, int accumulate,
                             cudaStream_t st);
// the same on the problems amap[0..Fa) of [F][nk] arrays only
rr_status launch_convert_d2f_map(int Fa, const int* amap, size_t nk, const double2* in,
                                 float2* out, cudaStream_t st);
rr_status launch_convert_f2d_map(int Fa, const int* amap, size_t nk, const float2* in,
                                 double2* out, int accumulate, cudaStream_t st);
// column 2-norms out[f][j] of x[f] ([F][N][k]); with amap only the problems
// amap[0..F) (F slots), the other entries of out untouched
rr_status launch_colnorm2(int F, int N, int k, const double2* x, double* part, int nblk,
                          double* out, cudaStream_t st, const int* amap = nullptr);
rr_status launch_gram(int F, int N, int k, const double2* Y, double2* part, int nblk,
                      double2* G, cudaStream_t st);
rr_status launch_cholesky(int F, int k, const double2* G, double2* R, double2* Rinv,
                          int* bad, double shift_rel, double* cond, cudaStream_t st);
// upper != 0: S is upper triangular (the kernel skips its zero lower part)
rr_status launch_right_mul(int F, int N, int k, const double2* Y, const double2* S,
                           double2* out, cudaStream_t st, int upper = 0);
rr_status launch_small_mul(int F, int k, const double2* A, const double2* B, double2* C,
                           cudaStream_t st);
rr_status launch_jacobi_svd(int F, int k, const double2* R, double* sigma, double2* Ul,
                            double2* Vr, int* sweeps, cudaStream_t st);
rr_status launch_col_scale(int F, int N, int k, const double2* in, const double* sigma,
                           double2* out, cudaStream_t st);
rr_status launch_finish_modes(int F, int N, int k, double2* U, double2* V, double* sigma,
                              double2* tmpU, double2* tmpV, double* part, int nblk,
                              int* rank, double2* phase, cudaStream_t st);

rr_status launch_axpy(size_t n, const double2* d, double2* x, cudaStream_t st);

// grad.cu: grad[3][nx*ny] += d(sum_f sum_{j<J} sigma_j^2)/d(rho, U, V) from the
// sandwich vectors A = A^{-H} W^{1/2} u, B = A^{-1} W^{-1/2} v ([F][N][J]);
// sigma [F][sstride]; featbar scratch [nx*ny][18].
rr_status launch_gain_grad(const OpDev& d, const rr_grid& g, int F, int J, const double2* A,
                           const double2* B, const double* sigma, int sstride, double* featbar,
                           double* grad, cudaStream_t st);

// prof.cu: launch counting and per-class event timing (classes of rr.h)
enum {
  PROF_SCHUR = 0, PROF_PANEL = 1, PROF_ROWBLOCK = 2, PROF_UPDATE = 3, PROF_FINALIZE = 4,
  PROF_SWEEP = 5, PROF_RESIDUAL = 6, PROF_GRAM = 7, PROF_RIGHTMUL = 8, PROF_SMALL = 9,
  PROF_INNER = 10, PROF_OTHER = 11, PROF_N = 12
};
// While a ProfSuspend lives (graph capture), launches are neither counted
// nor timed.
struct ProfSuspend {
  ProfSuspend();
  ~ProfSuspend();
};
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);
void prof_count(int n);
// bounded-wait diagnostics: polls before an mbarrier wait gives up, and
// whether the next tensor-core sweep launch stalls (test-only, rr_debug_waits)
uint32_t wait_tries();
int take_stall();

int num_sms(int device);
