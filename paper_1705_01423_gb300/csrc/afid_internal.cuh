// Internal definitions shared by the libafid translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "../../include/afid.h"
#include "fft.cuh"

namespace afid {

// Wall-normal metric, device resident (one allocation). Index ranges:
//   dzc, rdzc            [nz]     cell widths and their inverses
//   dzf, rdzf            [nz+1]   centre spacings; dzf[0] = dzc[0]/2, dzf[nz] = dzc[nz-1]/2
//   pa, pc               [nz]     Poisson operator (zero-flux walls): pa[0] = pc[nz-1] = 0
//   ca, cc               [nz]     cell operator with Dirichlet walls half a cell away
//   fa, fc               [nz+1]   face operator on interior faces k = 1..nz-1
//   wlo, whi             [nz+1]   volume weights of the cell->face interpolation
//                                 (dzc[k-1], dzc[k]) / (2 dzf[k]) on interior faces
//   pdiag                [nz]     pa + pc + 2/dx^2 + 2/dy^2
struct Metric {
  const double *dzc, *rdzc, *dzf, *rdzf, *pa, *pc, *ca, *cc, *fa, *fc, *wlo, *whi;
  const double* pdiag;  // [nz] pa + pc + 2/dx^2 + 2/dy^2 (minus the 7-point diagonal)
};

// Small device-resident scalars (one allocation).
enum Scalar {
  S_DT = 0,        // time step set by afid_cfl
  S_CFLM,          // last CFL number
  S_RHS_MEAN,      // weighted mean removed from the last rhs
  S_RHS_ABSMAX,    // max |rhs| of the last solve (as an ordered uint64 bit pattern)
  S_MAXDIV,        // max |div| (bit pattern)
  S_BNORM2,        // mixed: ||b - mean||_2^2
  S_RNORM2,        // mixed: ||r||_2^2 of the last residual
  S_BMEAN,         // mixed: weighted mean of b
  S_CONVERGED,     // mixed: 1.0 when converged
  S_ITERS,         // mixed: iterations done
  S_PROJ_S,        // projection scale s (alpha_l dt in a substep)
  S_PROJ_BETA,     // pressure-update coefficient beta
  S_DNORM2,        // mixed: ||delta||_2^2 of the last correction
  S_DPREV2,        // mixed: ||delta||_2^2 of the correction before it
  S_PHINORM2,      // mixed: ||phi||_2^2 after the last correction
  S_ERREST,        // mixed: estimated relative error of phi
  S_D1NORM2,       // mixed: ||d_1||^2 (the first correction, a proxy for ||phi||^2)
  S_PHIMEAN,       // mixed: weighted mean of phi after the last correction
  S_FAULT,         // 1.0 when a bounded wait inside a kernel gave up
  S_PROJ_RS,       // 1 / S_PROJ_S (formed once where S_PROJ_S is set)
  S_COUNT = 20
};

// Kernel families for the event-based instrumentation (afid_profile_*).
enum KFam {
  KF_R2C = 0,   // forward x transform (+ fused divergence)
  KF_FFTY,      // y transforms, forward and inverse
  KF_THOMAS,    // Thomas sweeps (incl. FP64 low modes)
  KF_ZERO,      // exact (0,0) mode
  KF_C2R,       // inverse x transform
  KF_PROJECT,   // projection / pressure update / divergence
  KF_RHS,       // RK3 explicit terms
  KF_CN,        // Crank-Nicolson sweeps
  KF_CFL,       // CFL reduction
  KF_REFINE,    // mixed-precision residual, norms, checks
  KF_ADJ,       // adjoint-only kernels
  KF_CNTAB,     // Crank-Nicolson factor tables (one tiny kernel per substep)
  KF_MR_PROLONG,   // refined temperature grid: velocity prolongation (+ time interpolation)
  KF_MR_RHS,       // refined temperature grid: explicit terms and right-hand side
  KF_MR_RESTRICT,  // refined temperature grid: restriction to the momentum grid
  KF_YT,           // mixed, small nz: fused y transforms + wall-normal solves
  KF_COUNT
};

struct Prof {
  bool on = false;
  bool overflow = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> fam;  // family of each recorded begin event
  int used = 0;          // events recorded (begin/end pairs)
  double ms[KF_COUNT] = {};
  long long n[KF_COUNT] = {};
};

// Arrays per variable set in the Crank-Nicolson table (k_cn_tables): sub,
// m, c', sup, and the explicit-side coefficients 2 beta a, 2 beta c,
// -2 beta (a + c); set 0 also carries the per-plane factors of the explicit
// terms: alpha_l dt / dzf, dzc^-1 / 4, dzf^-1 / 4 (arrays 7, 8, 9). Arrays
// 10-17 are the same coefficients multiplied by the row's reciprocal pivot
// m_k, so that the explicit-terms kernels write m_k R_k directly and the
// forward elimination is d'_k = m_k R_k - (m_k sub_k) d'_{k-1}: 10 m sub,
// 11-13 m times arrays 4-6, 14 m dt gamma_l, 15 m dt rho_l, 16 the pressure
// gradient factor times m (set 0: alpha_l dt / dx; set 1: alpha_l dt / dzf_k),
// 17 (set 0) m alpha_l dt / dy.
constexpr int CN_TAB_ARRAYS = 18;
enum CnTab {
  CN_SUB = 0, CN_M, CN_CP, CN_SUP, CN_EA, CN_EC, CN_ED, CN_PZ, CN_QZ, CN_QZF,
  CN_MSUB, CN_MEA, CN_MEC, CN_MED, CN_MCG, CN_MCR, CN_MGX, CN_MGY
};

struct Grid {
  int nx, ny, nz;
  int M;         // nx / 2
  int P;         // spectral row pitch in complex elements (>= M + 1)
  int nyh;       // ny / 2 + 1 (rows of the Thomas factor table)
  double dx, dy, rdx, rdy, rdx2, rdy2;
};

}  // namespace afid

struct afid_ctx {
  afid::Grid g;
  double lx, ly;
  double hz;  // sum of dzc over k = 0..nz-1 in that order (the wall-normal extent)
  int prec;
  double tol;
  int max_iter;
  int flags;
  afid_phys phys;
  cudaStream_t stream;
  int device;
  int num_sms;

  // metric
  void* metric_buf;
  afid::Metric m;
  // twiddle tables exp(-2 pi i m / N): x table of nx entries, y table of ny entries
  double2 *twx64, *twy64;
  float2 *twx32, *twy32;
  // FP64 y transform, power-of-two ny >= 64: tangent-form twiddle tables
  // (tan_tables), forward [0] and inverse [1], ytan_len doubles each; null
  // otherwise (the plain twiddles are used)
  double* ytan64[2];
  int ytan_len;
  // FP64 x transforms, power-of-two M = nx/2 >= 64: the same for the M-point
  // FFT (twiddles exp(-2 pi i m/M))
  double* xtan64[2];
  int xtan_len;
  // Thomas factor tables mtab[k][kyh][kx] (kyh = min(ky, ny-ky)); mtab64 always,
  // mtab32 in mixed mode; low-mode mask threshold for mixed mode
  double* mtab64;
  float* mtab32;
  // mixed, small nz (fuse_yt): the FP32 table transposed to [kx][k][kyh] for
  // the fused y-transform / Thomas kernel, its launch shape
  float* mtabt32;
  int fuse_yt, yt_threads, yt_lmax;  // yt_lmax: most low modes in one kx column
  int warp_tridiag;  // FP64: the warp-partitioned solver for every system (flag or auto)
  size_t yt_smem;
  double lam_thr;
  double* lamx;  // [M+1]
  double* lamy;  // [nyh]
  // spectral workspace [nz][ny][P] complex (double2 in FP64, float2 in mixed)
  void* spec;
  // physical workspace
  double* phi;    // [nz][ny][nx]
  double* bbuf;   // mixed: FP64 right-hand side kept for the residual [nz][ny][nx]
  double* R[4];   // substep right-hand sides (u, v: cells; w, T: faces)
  double* cntab;  // Crank-Nicolson factor tables [3][CN_TAB_ARRAYS][nz+1]
  // mixed precision: FP32 copies of the Poisson off-diagonals; the low modes
  // solved in FP64 by the warp solver: their list (ky, kx) and a mask
  // lowslot[ky][kx] (>= 0 for a low mode) that the FP32 sweep skips
  float *pa32, *pc32;
  int* lowslot;
  int2* low_modes;
  int nlow;
  double2* low_scratch;
  double* scal;   // device scalars (Scalar enum)
  double* part;   // reduction partials
  int part_len;
  double* part2;  // mixed: per-block (||delta||^2, sum dzc delta) of the accumulate pass
  int part2_len;
  double* part3;  // mixed: per-block partials of the forward pass (stats of b / ||r||^2)
  // mixed: the last residual as a two-float (head, tail) pair, the last FP32
  // correction added to phi, and two-float splits of pa, pc, pdiag ([3][nz])
  // for the residual update r_k = r_{k-1} - L delta_{k-1}
  float2* rres;
  float* dprev;
  float2* cff;
  // wall-normal statistics: profiles [nz+1][AFID_STAT_NQ] and 8 scalars
  double* stat_buf;
  // host copy of the nz+1 face coordinates (refined grids are built from it)
  double* zf_host;
  size_t bytes;
  long long launches;
  afid::Prof* prof;
  // TMA-staged FP32 y transforms: tensor map of the spectral workspace and
  // launch shape and tile width (kx columns); tma_y = 0 when unused (FP64
  // contexts, ny not a power of two or > 2048, AFID_NO_TMA)
  CUtensorMap tmy;
  int tma_y;
  int tmy_stages, tmy_threads, tmy_blocks_per_sm, tmy_tk;
  int tma_stall_once;  // test of the timeout path: the next TMA launch stalls block 0
  size_t tmy_smem;
};

namespace afid {

// Host wall-normal metric of the faces zf[0..nz]: the METRIC_ARRAYS arrays of
// Metric, in its order, each nz+1 long (unused tail entries zero), written to
// out[a (nz+1) + k] without any allocation (the allocation-free solve fills a
// static staging buffer with it); metric_host returns the same in `flat` with
// the offsets of the arrays in `offs`; metric_view is the device view of an
// uploaded copy.
constexpr int METRIC_ARRAYS = 13;
void metric_fill(int nz, double rdx2, double rdy2, const double* zf, double* out);
void metric_host(int nz, double rdx2, double rdy2, const double* zf, std::vector<double>& flat,
                 std::vector<size_t>& offs);
// exp(-2 pi i m / N) as (c, s), evaluated in the first octant and mapped by
// symmetry (the FFT twiddle tables)
void twiddle(long long m, long long N, double& c, double& s);
// modified wavenumber of the periodic 3-point second difference (Sec. 2.2):
// 4 sin^2(pi k / n) / h^2
double mod_wavenumber(int k, int n, double h);
Metric metric_view(const double* dev, const std::vector<size_t>& offs);

// launchers (stream-ordered; return cudaError_t of the launch)
cudaError_t init_thomas_tables(afid_ctx* c);
// TMA y transform of the FP32 (mixed-precision) spectral passes: set-up at
// create, launch
cudaError_t init_ffty_tma(afid_ctx* c);
template <typename R>
cudaError_t run_fft_y_tma(afid_ctx* c, const typename cplx<R>::T* tw, bool inv, const double* skip);
// Direct FP64 solve of L phi = src / s, src = rhs (rhs != NULL) or D(u, v, w);
// s is read from the device scalar S_PROJ_S when `dev_s`, else 1.
cudaError_t spectral_solve(afid_ctx* c, const double* rhs, const double* u, const double* v,
                           const double* w, bool dev_s, double* phi, bool want_stats);
int tan_tables(int N, const double2* tw, bool inv, double* out);  // host; k_spectral.cu
int c2r_blocks(const Grid& g);
// Fused small-nz kernel (mixed): shared memory (lmax: most low modes in one
// kx column) and threads per block.
size_t yfft_thomas32_smem(const Grid& g, int lmax);
int yfft_thomas32_threads(const Grid& g);
// Sets c->fuse_yt (and the attributes of the fused kernel) when the brick of
// one kx column, its pivots and its low modes fit in shared memory and the
// FP32 spectral array fits in half of L2.
cudaError_t init_yfft_thomas32(afid_ctx* c, int lmax);
// Mixed-precision refined solve of L phi = b (FP64 b, resident) into phi.
cudaError_t mixed_solve(afid_ctx* c, const double* b, double* phi, bool stats);
// One FP32 spectral solve of refinement step `it`: b (it = 0), the FP64
// residual (b - mean) - L phi_in (it = 1) or the residual update
// r - L delta_prev in two-float arithmetic (it >= 2), formed in the forward
// transform; phi = delta (it = 0) or phi += delta - mean_W(phi).
cudaError_t spectral_solve_fp32(afid_ctx* c, const double* b, const double* phi_in, double* phi,
                                const double* skip, int it, bool stats);
// Reduction of the stats of b taken by the first forward transform.
cudaError_t bstats_final(afid_ctx* c);
// Wall-normal statistics of (u, v, w, T) into c->stat_buf (profiles, then the
// scalars of afid_stats).
cudaError_t statistics(afid_ctx* c, const double* u, const double* v, const double* w, const double* T);
// The same for any grid and metric (profiles [nz+1][AFID_STAT_NQ], then 8
// scalars, into stat_buf).
cudaError_t statistics_grid(const Grid& g, const Metric& m, const afid_phys& ph, const double* u,
                            const double* v, const double* w, const double* T, double* stat_buf,
                            cudaStream_t st);
// Volume Nusselt number 1 + coef <w T>_V into c->stat_buf[nz + 1] and, for
// non-NULL gw / gT, its derivatives with respect to w and T.
cudaError_t nusselt(afid_ctx* c, const double* w, const double* T, double coef, double* gw,
                    double* gT);
// b = D(u, v, w) / s (s from S_PROJ_S)
cudaError_t divergence_to(afid_ctx* c, const double* u, const double* v, const double* w, double* b);
// projection with s, beta read from S_PROJ_S / S_PROJ_BETA
cudaError_t project(afid_ctx* c, double* u, double* v, double* w, double* p, const double* phi);
cudaError_t set_proj_scalars(afid_ctx* c, double s, double beta);
cudaError_t max_divergence(afid_ctx* c, const double* u, const double* v, const double* w,
                           double* out_dev);
cudaError_t cfl(afid_ctx* c, const double* u, const double* v, const double* w, double cfl,
                double dt_max, double* cflm_dev);
cudaError_t rk3_explicit(afid_ctx* c, int l, double dt, const double* u, const double* v,
                         const double* w, const double* T, const double* p, double* Hu,
                         double* Hv, double* Hw, double* HT);
cudaError_t cn_tables(afid_ctx* c, int l, double dt);
cudaError_t cn_sweeps(afid_ctx* c, double* u, double* v, double* w, double* T);
cudaError_t scale_cells(afid_ctx* c, const double* in, double* out, bool forward);
// The Crank-Nicolson tables of substep l for any grid and metric (into tab,
// with the substep scalars in scal), and the forward sweep of the temperature
// operator alone: T += A^-1 RT on the interior faces (RT overwritten).
cudaError_t cn_tables_grid(const Grid& g, const Metric& m, int l, double dt, double* scal, double nu,
                           double kappa, double* tab, cudaStream_t st);
cudaError_t cn_sweep_scalar(const Grid& g, const double* tab, double* RT, double* T, cudaStream_t st);
cudaError_t adjoint_explicit(afid_ctx* c, int l, double dt, const double* u, const double* v,
                             const double* w, const double* T, double* gu, double* gv,
                             double* gw, double* gT, double* gp, double* gHu, double* gHv,
                             double* gHw, double* gHT);
// R_q = A_q^-T g_q for the four Crank-Nicolson operators (g_q unchanged)
cudaError_t cn_sweeps_adjoint(afid_ctx* c, double* gu, double* gv, double* gw, double* gT);
cudaError_t project_adjoint_pre(afid_ctx* c, double* gu, double* gv, double* gw, const double* gp,
                                double s, double beta);
cudaError_t project_adjoint_post(afid_ctx* c, double* gu, double* gv, double* gw, double* gp,
                                 const double* psi, double s, double beta);

// RK3 coefficients (Sec. 2.1, low-storage set): gamma, rho, alpha = gamma + rho
__host__ __device__ inline double rk_gamma(int l) { return l == 0 ? 8.0 / 15.0 : (l == 1 ? 5.0 / 12.0 : 3.0 / 4.0); }
__host__ __device__ inline double rk_rho(int l) { return l == 0 ? 0.0 : (l == 1 ? -17.0 / 60.0 : -5.0 / 12.0); }
__host__ __device__ inline double rk_alpha(int l) { return rk_gamma(l) + rk_rho(l); }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Brackets the launches of one kernel family with CUDA events on the context's
// stream when instrumentation is on (no effect otherwise).
struct ProfScope {
  afid_ctx* c;
  int fam;
  bool rec;
  ProfScope(afid_ctx* ctx, int f) : c(ctx), fam(f), rec(false) {
    Prof* p = c->prof;
    if (p && p->on && p->used + 2 <= (int)p->ev.size()) {
      cudaEventRecord(p->ev[p->used], c->stream);
      p->fam[p->used / 2] = fam;
      rec = true;
    } else if (p && p->on) {
      p->overflow = true;
    }
  }
  ~ProfScope() {
    if (rec) {
      Prof* p = c->prof;
      cudaEventRecord(p->ev[p->used + 1], c->stream);
      p->used += 2;
    }
  }
};

// Periodic neighbours of index i in [0, n) (any n; the grid sizes are
// 2^a 3^b 5^c).
__host__ __device__ __forceinline__ int wrap_next(int i, int n) { return i + 1 < n ? i + 1 : 0; }
__host__ __device__ __forceinline__ int wrap_prev(int i, int n) { return i > 0 ? i - 1 : n - 1; }
// i + d for 0 <= i < n, |d| < n
__host__ __device__ __forceinline__ int wrap_add(int i, int d, int n) {
  const int j = i + d;
  return j >= n ? j - n : (j < 0 ? j + n : j);
}

inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Largest block width in x among {128, 64, 32, 16} that divides nx and is
// at most `cap` (nx is a multiple of 16).
inline int x_block(int nx, int cap) {
  for (int b = 128; b >= 16; b /= 2)
    if (b <= cap && nx % b == 0) return b;
  return 16;
}

// s += x with the exact rounding error of the addition (Knuth's TwoSum, with
// round-to-nearest intrinsics so that no step is contracted or re-associated)
// added to the compensation c; s + c is the compensated sum.
__device__ __forceinline__ void two_sum_acc(double& s, double& c, double x) {
  const double t = __dadd_rn(s, x);
  const double xp = __dsub_rn(t, s);
  const double e = __dadd_rn(__dsub_rn(s, __dsub_rn(t, xp)), __dsub_rn(x, xp));
  s = t;
  c = __dadd_rn(c, e);
}

// Ordered bit pattern of a non-negative double for atomicMax.
__device__ __forceinline__ unsigned long long dbl_key(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

}  // namespace afid
