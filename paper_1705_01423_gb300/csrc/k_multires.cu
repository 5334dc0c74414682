// Multiple-resolution temperature grid (Sec. 6, conclusions and future
// plans): the temperature lives on a grid refined rx x ry x rz times over the
// momentum grid and is advanced with its own refined RK3 / Crank-Nicolson
// steps; the momentum sees its restriction as buoyancy.
//
// Fine grid: every coarse cell split into rx x ry x rz equal cells, the fine
// z-faces nesting the coarse ones (coarse face k = fine face rz k).
// One refined substep (all FP64; bound by the FP64 issue rate of this part,
// like the rest of the library):
//   k_mr_lerp        coarse velocity at the substep's start time, linear in
//                    time between the coarse states at t and t + dt (skipped
//                    when that time is t);
//   k_mr_prolong_sep trilinear prolongation of each velocity component from
//                    its coarse staggered positions to its fine ones, one
//                    thread per fine (x, y) column walking up in z: a block's
//                    x-interpolated coarse rows are formed once per coarse
//                    plane in shared memory, and the bilinear value of a plane
//                    serves every fine level between that plane and the next
//                    (k_mr_prolong: the per-column form, for fine widths that
//                    are not multiples of 32);
//   k_mr_scalar_rhs_sh  explicit terms (advection in divergence form,
//                    horizontal diffusion) and the Crank-Nicolson right-hand
//                    side of the temperature, the single-grid equation on the
//                    fine grid, with the x/y face fluxes shared between
//                    neighbouring threads (k_mr_scalar_rhs: per column);
//   k_cn_tables, k_cn_sweep  the fine grid's factors and the T sweep.
// k_mr_restrict averages the fine temperature over each coarse cell's
// horizontal extent on the coincident face plane; afid_mr_statistics runs the
// wall-normal statistics on the fine grid.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "afid_internal.cuh"

using namespace afid;

// Index / weight tables of the prolongation: for every fine index the lower
// coarse sample and the weight of the upper one.
enum MrTable { T_XF = 0, T_XC, T_YF, T_YC, T_ZC, T_ZF, T_COUNT };

struct afid_mr {
  afid_ctx* c;
  int r[3];
  Grid gf;
  void* metric_buf;
  Metric mf;
  int* itab;
  double* wtab;
  size_t off[T_COUNT];
  double* cntab;  // fine-grid Crank-Nicolson tables [3][CN_TAB_ARRAYS][nzf+1]
  double* scal;   // fine-grid substep scalars
  double *uf, *vf, *wf;  // fine velocity
  double *HT, *RT;       // fine explicit terms and right-hand side (faces)
  double *u0, *v0, *w0;  // coarse velocity at the start of a coupled step
  double *ul, *vl, *wl;  // coarse velocity at an intermediate time
  double* Tc;            // restricted temperature (coarse faces)
  double* stat_buf;      // fine-grid statistics: profiles [nzf+1][AFID_STAT_NQ], 8 scalars
  size_t bytes;
};

namespace afid {
namespace {

struct MrTab {
  const int *ix, *iy, *iz;
  const double *wx, *wy, *wz;
};

// out = trilinear prolongation of q. CELL: q is a cell field [nz][ny][nx],
// extended along z by the wall values qbot, qtop (extended index e: 0 bottom
// wall, 1..nz the planes 0..nz-1, nz+1 top wall), fine levels K = 0..nzf-1;
// otherwise q is a face field [nz+1][ny][nx], fine levels K = 0..nzf.
// The table index of a fine level depends on K only, so the refresh branch
// is uniform over the block.
template <bool CELL>
__global__ void __launch_bounds__(256) k_mr_prolong(Grid gc, Grid gf, MrTab t,
                                                    const double* __restrict__ q, double qbot,
                                                    double qtop, double* __restrict__ out, int kchunk) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= gf.nx || Y >= gf.ny) return;
  const int nx = gc.nx, ny = gc.ny;
  const size_t NXYc = (size_t)nx * ny, NXYf = (size_t)gf.nx * gf.ny;
  const int i0 = t.ix[X], i1 = wrap_next(i0, nx);
  const int j0 = t.iy[Y], j1 = wrap_next(j0, ny);
  const double wx = t.wx[X], wy = t.wy[Y];
  const size_t a00 = (size_t)j0 * nx + i0, a01 = (size_t)j0 * nx + i1;
  const size_t a10 = (size_t)j1 * nx + i0, a11 = (size_t)j1 * nx + i1;
  auto plane = [&](int kc) {
    const double* p = q + (size_t)kc * NXYc;
    const double lo = fma(wx, p[a01] - p[a00], p[a00]);
    const double hi = fma(wx, p[a11] - p[a10], p[a10]);
    return fma(wy, hi - lo, lo);
  };
  auto ext = [&](int e) -> double {
    if (CELL) return e == 0 ? qbot : (e == gc.nz + 1 ? qtop : plane(e - 1));
    return plane(e);
  };
  const int nK = CELL ? gf.nz : gf.nz + 1;
  const int K0 = blockIdx.z * kchunk, K1 = min(nK, K0 + kchunk);
  const size_t col = (size_t)Y * gf.nx + X;
  int cur = -2;
  double lo = 0.0, hi = 0.0;
  for (int K = K0; K < K1; ++K) {
    const int e = t.iz[K];
    if (e != cur) {
      lo = e == cur + 1 ? hi : ext(e);
      hi = ext(e + 1);
      cur = e;
    }
    out[(size_t)K * NXYf + col] = fma(t.wz[K], hi - lo, lo);
  }
}

// The same prolongation for blocks of 32 x 8 fine columns (nx_f a multiple
// of 32, ny_f of 8): the x interpolation of the coarse rows the block needs
// (at most MR_ROWS of them) is formed once per coarse plane in shared memory
// and shared by the fine rows between them, then each thread interpolates in
// y and z. Per fine column and coarse plane: one y interpolation plus its
// share of the x interpolations (about 2/ry + 1/4 of one), against three.
// Every branch on the plane index is uniform over the block (the tables
// depend on K only), so the barriers inside it are reached by all threads.
constexpr int MR_ROWS = 10;
template <bool CELL>
__global__ void __launch_bounds__(256) k_mr_prolong_sep(Grid gc, Grid gf, MrTab t,
                                                        const double* __restrict__ q, double qbot,
                                                        double qtop, double* __restrict__ out, int kchunk) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int X = blockIdx.x * 32 + tx, Y = blockIdx.y * 8 + ty;
  const int nx = gc.nx, ny = gc.ny;
  const size_t NXYc = (size_t)nx * ny, NXYf = (size_t)gf.nx * gf.ny;
  __shared__ double xr[2][MR_ROWS][32];
  // coarse rows of the block: jr0, jr0 + 1, ... (mod ny); this thread's two
  const int jr0 = t.iy[blockIdx.y * 8];
  int nrows = t.iy[blockIdx.y * 8 + 7] - jr0;
  if (nrows < 0) nrows += ny;
  nrows += 2;
  int r0 = t.iy[Y] - jr0;
  if (r0 < 0) r0 += ny;
  const double wy = t.wy[Y];
  // the x-interpolation task of this thread: (row, column) pairs tid, tid + 256
  const int nx_tasks = nrows * 32;
  // Bilinear value of coarse plane kc. The two buffers alternate between
  // calls, so a buffer is rewritten only after the barrier of the call in
  // between, which every thread reaches after reading it.
  int b = 0;
  auto plane = [&](int kc) {
    const double* p = q + (size_t)kc * NXYc;
    for (int a = tid; a < nx_tasks; a += 256) {
      const int row = a >> 5, xc = a & 31;
      int jr = jr0 + row;
      if (jr >= ny) jr -= ny;
      const int Xa = blockIdx.x * 32 + xc;
      const int i0 = t.ix[Xa], i1 = wrap_next(i0, nx);
      const double* pr = p + (size_t)jr * nx;
      xr[b][row][xc] = fma(t.wx[Xa], pr[i1] - pr[i0], pr[i0]);
    }
    __syncthreads();
    const double lo = xr[b][r0][tx], hi = xr[b][r0 + 1][tx];
    b ^= 1;
    return fma(wy, hi - lo, lo);
  };
  auto ext = [&](int e) -> double {
    if (CELL) return e == 0 ? qbot : (e == gc.nz + 1 ? qtop : plane(e - 1));
    return plane(e);
  };
  const int nK = CELL ? gf.nz : gf.nz + 1;
  const int K0 = blockIdx.z * kchunk, K1 = min(nK, K0 + kchunk);
  const size_t col = (size_t)Y * gf.nx + X;
  int cur = -2;
  double lo = 0.0, hi = 0.0;
  for (int K = K0; K < K1; ++K) {
    const int e = t.iz[K];
    if (e != cur) {  // uniform: e depends on K only
      lo = e == cur + 1 ? hi : ext(e);
      hi = ext(e + 1);
      cur = e;
    }
    out[(size_t)K * NXYf + col] = fma(t.wz[K], hi - lo, lo);
  }
}

// out_f = a_f + theta (b_f - a_f) for the three coarse velocity fields
// (blockIdx.y = component; u, v: n cells, w: n + NXY faces).
__global__ void k_mr_lerp(size_t n, size_t nxy, double theta, const double* __restrict__ a0,
                          const double* __restrict__ a1, const double* __restrict__ a2,
                          const double* __restrict__ b0, const double* __restrict__ b1,
                          const double* __restrict__ b2, double* __restrict__ o0,
                          double* __restrict__ o1, double* __restrict__ o2) {
  const int f = blockIdx.y;
  const double* a = f == 0 ? a0 : (f == 1 ? a1 : a2);
  const double* b = f == 0 ? b0 : (f == 1 ? b1 : b2);
  double* o = f == 0 ? o0 : (f == 1 ? o1 : o2);
  const size_t len = f == 2 ? n + nxy : n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    o[i] = fma(theta, b[i] - a[i], a[i]);
}

// Coarse face temperature = mean of the rx x ry fine values of face plane rz k.
__global__ void k_mr_restrict(Grid gc, Grid gf, int rx, int ry, int rz, const double* __restrict__ Tf,
                              double* __restrict__ Tc) {
  const size_t NXYc = (size_t)gc.nx * gc.ny, NXYf = (size_t)gf.nx * gf.ny;
  const size_t total = NXYc * (gc.nz + 1);
  const double rn = 1.0 / (double)(rx * ry);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / NXYc);
    const size_t rem = idx - (size_t)k * NXYc;
    const int j = (int)(rem / gc.nx), i = (int)(rem - (size_t)j * gc.nx);
    const double* p = Tf + (size_t)rz * k * NXYf + (size_t)ry * j * gf.nx + (size_t)rx * i;
    double s = 0.0;
    for (int a = 0; a < ry; ++a)
      for (int b = 0; b < rx; ++b) s += p[(size_t)a * gf.nx + b];
    Tc[idx] = s * rn;
  }
}

// Temperature explicit terms H and right-hand side R of RK3 substep l on the
// fine grid (faces k = 1..nz-1; H = 0 on the walls):
//   H = -[(F^x_i+1 - F^x_i)/dx + (F^y_j+1 - F^y_j)/dy + (F^z_k - F^z_k-1)/dzf_k]
//       + kappa (dxx + dyy) T,
//   F^x_i = uf_i (T_i-1 + T_i)/2, uf = (dzc_k-1 u_k-1 + dzc_k u_k)/(2 dzf_k) on
//   face k (y likewise), F^z at cell k = (w_k + w_k+1)(T_k + T_k+1)/4;
//   R = dt [gamma_l H + rho_l Hprev] + alpha_l dt kappa dzz T.
// One thread per (x, y) column, walking up in k and carrying the z flux, the
// lower-plane velocities and the three T values of the column.
// Scalar factors of the temperature terms, formed on the host (as kernel
// parameters they sit in the constant bank, read directly by the FMAs): 1/2 of
// the inverse spacings and the horizontal diffusion weights with kappa folded
// in, kappa/dx^2, kappa/dy^2, 2 kappa (1/dx^2 + 1/dy^2).
struct ScalarW {
  double hx, hy, krx, kry, kl0;
};

__global__ void __launch_bounds__(256) k_mr_scalar_rhs(Grid g, Metric m, ScalarW sw, int l, double dt,
                                                       const double* __restrict__ u,
                                                       const double* __restrict__ v,
                                                       const double* __restrict__ w,
                                                       const double* __restrict__ T,
                                                       double* __restrict__ HT, double* __restrict__ RT,
                                                       const double* __restrict__ cnt, int kchunk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, nz = g.nz;
  const size_t NXY = (size_t)nx * g.ny;
  const int ip = wrap_next(i, nx), im = wrap_prev(i, nx);
  const int jp = wrap_next(j, g.ny), jm = wrap_prev(j, g.ny);
  const size_t col = (size_t)j * nx + i;
  const size_t cip = (size_t)j * nx + ip, cim = (size_t)j * nx + im;
  const size_t cjp = (size_t)jp * nx + i, cjm = (size_t)jm * nx + i;
  const int L = nz + 1;
  // R is written multiplied by the reciprocal pivot of its Crank-Nicolson row:
  // the coefficients come pre-scaled per plane (set 2 of the fine-grid table)
  const double* __restrict__ mcg = cnt + (size_t)(2 * CN_TAB_ARRAYS + CN_MCG) * L;
  const double* __restrict__ mcr = cnt + (size_t)(2 * CN_TAB_ARRAYS + CN_MCR) * L;
  (void)dt;
  const double hx = sw.hx, hy = sw.hy;
  const double* __restrict__ ea = cnt + (size_t)(2 * CN_TAB_ARRAYS + CN_MEA) * L;  // m alpha dt kappa dzz
  const double* __restrict__ ec = ea + L;
  const double* __restrict__ ed = ec + L;
  const double* __restrict__ qzf = cnt + (size_t)CN_QZF * L;  // dzf^-1 / 4

  const int kb = blockIdx.z * kchunk;
  const int k0 = max(1, kb), k1 = min(nz, kb + kchunk);
  if (blockIdx.z == 0) {
    HT[col] = 0.0;
    HT[(size_t)nz * NXY + col] = 0.0;
  }
  if (k0 >= k1) return;
  // column state below face k0: cell k0-1 and face k0
  size_t c = (size_t)(k0 - 1) * NXY;
  double ukm = u[c + col], uipkm = u[c + cip], vkm = v[c + col], vjpkm = v[c + cjp];
  double tkm = T[c + col], wkm = w[c + col];
  double t0 = T[c + NXY + col], w0 = w[c + NXY + col];
  double fz0 = (wkm + w0) * (tkm + t0);
  for (int k = k0; k < k1; ++k) {
    c = (size_t)k * NXY;
    const double uk = u[c + col], uipk = u[c + cip], vk = v[c + col], vjpk = v[c + cjp];
    const double tk1 = T[c + NXY + col], wk1 = w[c + NXY + col];
    const double tip = T[c + cip], tim = T[c + cim], tjp = T[c + cjp], tjm = T[c + cjm];
    const double wlo = m.wlo[k], whi = m.whi[k];
    const double ufi = fma(wlo, ukm, whi * uk), ufip = fma(wlo, uipkm, whi * uipk);
    const double vfj = fma(wlo, vkm, whi * vk), vfjp = fma(wlo, vjpkm, whi * vjpk);
    const double fx0 = ufi * (tim + t0), fx1 = ufip * (t0 + tip);
    const double fy0 = vfj * (tjm + t0), fy1 = vfjp * (t0 + tjp);
    const double fz1 = (w0 + wk1) * (t0 + tk1);
    const double A = fma(fz1 - fz0, qzf[k], fma(fy1 - fy0, hy, (fx1 - fx0) * hx));
    const double H = fma(sw.krx, tip + tim, fma(sw.kry, tjp + tjm, fma(-sw.kl0, t0, -A)));
    const double z = fma(ea[k], tkm, fma(ec[k], tk1, ed[k] * t0));
    double r = fma(mcg[k], H, z);
    if (l > 0) r = fma(mcr[k], HT[c + col], r);
    HT[c + col] = H;
    RT[c + col] = r;
    ukm = uk;
    uipkm = uipk;
    vkm = vk;
    vjpkm = vjpk;
    tkm = t0;
    t0 = tk1;
    w0 = wk1;
    fz0 = fz1;
  }
}

// The same terms with the x and y face fluxes shared between neighbours
// (blocks of BY rows of 32 WPR points; nx a multiple of 32 WPR, ny of BY).
// Each thread forms the flux through its own left (x) and lower (y) face;
// the right-face flux comes from the next lane (shuffle), across the two warps
// of a 64-wide row through shared memory, and is formed directly only at the
// block's right edge; the upper-face flux comes from the next row through a
// double-buffered shared array (one barrier per k), formed directly only in
// the block's last row. Masked lanes cost the same issue slots, so an edge
// branch costs its warp the full instruction count: wider blocks have fewer.
template <int BY, int WPR>
__global__ void __launch_bounds__(32 * WPR * BY, 2) k_mr_scalar_rhs_sh(
    Grid g, Metric m, ScalarW sw, int l, double dt, const double* __restrict__ u,
    const double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ T,
    double* __restrict__ HT, double* __restrict__ RT, const double* __restrict__ cnt, int kchunk) {
  constexpr int BX = 32 * WPR;
  constexpr unsigned FULL = 0xffffffffu;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * BX + tx, j = blockIdx.y * BY + ty;
  const int nx = g.nx, nz = g.nz;
  const size_t NXY = (size_t)nx * g.ny;
  const int ip = wrap_next(i, nx), im = wrap_prev(i, nx);
  const int jp = wrap_next(j, g.ny), jm = wrap_prev(j, g.ny);
  const size_t col = (size_t)j * nx + i;
  const size_t cip = (size_t)j * nx + ip, cim = (size_t)j * nx + im;
  const size_t cjp = (size_t)jp * nx + i, cjm = (size_t)jm * nx + i;
  const int L = nz + 1;
  // R is written multiplied by the reciprocal pivot of its Crank-Nicolson row:
  // the coefficients come pre-scaled per plane (set 2 of the fine-grid table)
  const double* __restrict__ mcg = cnt + (size_t)(2 * CN_TAB_ARRAYS + CN_MCG) * L;
  const double* __restrict__ mcr = cnt + (size_t)(2 * CN_TAB_ARRAYS + CN_MCR) * L;
  (void)dt;
  const double hx = sw.hx, hy = sw.hy;
  const double* __restrict__ ea = cnt + (size_t)(2 * CN_TAB_ARRAYS + CN_MEA) * L;
  const double* __restrict__ ec = ea + L;
  const double* __restrict__ ed = ec + L;
  const double* __restrict__ qzf = cnt + (size_t)CN_QZF * L;
  const bool last_x = tx == BX - 1, last_row = ty == BY - 1;
  __shared__ double sfy[2][BY][BX];  // lower-face y flux of every thread
  __shared__ double sfx[2][BY];      // left-face x flux of x = 32 (second warp of a row)

  const int kb = blockIdx.z * kchunk;
  const int k0 = max(1, kb), k1 = min(nz, kb + kchunk);
  if (blockIdx.z == 0) {
    HT[col] = 0.0;
    HT[(size_t)nz * NXY + col] = 0.0;
  }
  if (k0 >= k1) return;  // uniform over the block
  size_t c = (size_t)(k0 - 1) * NXY;
  double ukm = u[c + col], vkm = v[c + col];
  double tkm = T[c + col], wkm = w[c + col];
  double t0 = T[c + NXY + col], w0 = w[c + NXY + col];
  double fz0 = (wkm + w0) * (tkm + t0);
  for (int k = k0; k < k1; ++k) {
    c = (size_t)k * NXY;
    const int buf = k & 1;
    const double uk = u[c + col], vk = v[c + col];
    const double tk1 = T[c + NXY + col], wk1 = w[c + NXY + col];
    const double tip = T[c + cip], tim = T[c + cim], tjp = T[c + cjp], tjm = T[c + cjm];
    const double wlo = m.wlo[k], whi = m.whi[k];
    const double fxl = fma(wlo, ukm, whi * uk) * (tim + t0);
    const double fyb = fma(wlo, vkm, whi * vk) * (tjm + t0);
    sfy[buf][ty][tx] = fyb;
    if (WPR == 2 && tx == 32) sfx[buf][ty] = fxl;
    __syncthreads();
    double fxr = __shfl_down_sync(FULL, fxl, 1);
    if (WPR == 2 && tx == 31) fxr = sfx[buf][ty];
    if (__any_sync(FULL, last_x)) {
      if (last_x) fxr = fma(wlo, u[c - NXY + cip], whi * u[c + cip]) * (t0 + tip);
    }
    double fyt;
    if (last_row)  // the whole warp (one row) takes this branch
      fyt = fma(wlo, v[c - NXY + cjp], whi * v[c + cjp]) * (t0 + tjp);
    else
      fyt = sfy[buf][ty + 1][tx];
    const double fz1 = (w0 + wk1) * (t0 + tk1);
    const double A = fma(fz1 - fz0, qzf[k], fma(fyt - fyb, hy, (fxr - fxl) * hx));
    const double H = fma(sw.krx, tip + tim, fma(sw.kry, tjp + tjm, fma(-sw.kl0, t0, -A)));
    const double z = fma(ea[k], tkm, fma(ec[k], tk1, ed[k] * t0));
    double r = fma(mcg[k], H, z);
    if (l > 0) r = fma(mcr[k], HT[c + col], r);
    HT[c + col] = H;
    RT[c + col] = r;
    ukm = uk;
    vkm = vk;
    tkm = t0;
    t0 = tk1;
    w0 = wk1;
    fz0 = fz1;
  }
}

// z chunking so that a launch has about sixteen 256-thread blocks per SM
int z_chunk(const afid_ctx* c, long long blocks_per_plane, int levels) {
  const long long want = 16LL * c->num_sms;
  int nch = (int)((want + blocks_per_plane - 1) / blocks_per_plane);
  const int max_ch = levels / 16 > 0 ? levels / 16 : 1;
  nch = std::max(1, std::min(nch, max_ch));
  return (levels + nch - 1) / nch;
}

MrTab tables_for(const afid_mr* mr, int comp) {
  const int* I = mr->itab;
  const double* W = mr->wtab;
  const MrTable tx = comp == 0 ? T_XF : T_XC, ty = comp == 1 ? T_YF : T_YC, tz = comp == 2 ? T_ZF : T_ZC;
  return MrTab{I + mr->off[tx], I + mr->off[ty], I + mr->off[tz],
               W + mr->off[tx], W + mr->off[ty], W + mr->off[tz]};
}

cudaError_t prolong(afid_mr* mr, const double* u, const double* v, const double* w, double* uf,
                    double* vf, double* wf) {
  afid_ctx* c = mr->c;
  ProfScope ps(c, KF_MR_PROLONG);
  const Grid& gf = mr->gf;
  dim3 blk(32, 8);
  const long long bpp = (long long)ceil_div(gf.nx, 32) * ceil_div(gf.ny, 8);
  const int kc_c = z_chunk(c, bpp, gf.nz), kc_f = z_chunk(c, bpp, gf.nz + 1);
  dim3 gc_(ceil_div(gf.nx, 32), ceil_div(gf.ny, 8), ceil_div(gf.nz, kc_c));
  dim3 gf_(ceil_div(gf.nx, 32), ceil_div(gf.ny, 8), ceil_div(gf.nz + 1, kc_f));
  // shared x interpolation when the 32 x 8 blocks tile the fine plane (the
  // rows a block needs: at most 8/ry + 2 <= MR_ROWS)
  if (gf.nx % 32 == 0 && gf.ny % 8 == 0) {
    k_mr_prolong_sep<true><<<gc_, blk, 0, c->stream>>>(c->g, gf, tables_for(mr, 0), u, c->phys.u_bot,
                                                       c->phys.u_top, uf, kc_c);
    k_mr_prolong_sep<true><<<gc_, blk, 0, c->stream>>>(c->g, gf, tables_for(mr, 1), v, 0.0, 0.0, vf, kc_c);
    k_mr_prolong_sep<false><<<gf_, blk, 0, c->stream>>>(c->g, gf, tables_for(mr, 2), w, 0.0, 0.0, wf, kc_f);
  } else {
    k_mr_prolong<true><<<gc_, blk, 0, c->stream>>>(c->g, gf, tables_for(mr, 0), u, c->phys.u_bot,
                                                   c->phys.u_top, uf, kc_c);
    k_mr_prolong<true><<<gc_, blk, 0, c->stream>>>(c->g, gf, tables_for(mr, 1), v, 0.0, 0.0, vf, kc_c);
    k_mr_prolong<false><<<gf_, blk, 0, c->stream>>>(c->g, gf, tables_for(mr, 2), w, 0.0, 0.0, wf, kc_f);
  }
  c->launches += 3;
  return cudaGetLastError();
}

// fine velocity at t + theta dt (theta = 0: vel0 itself)
cudaError_t velocity_at(afid_mr* mr, double theta, const double* u0, const double* v0, const double* w0,
                        const double* u1, const double* v1, const double* w1, double* uf, double* vf,
                        double* wf) {
  if (theta == 0.0) return prolong(mr, u0, v0, w0, uf, vf, wf);
  if (theta == 1.0) return prolong(mr, u1, v1, w1, uf, vf, wf);
  afid_ctx* c = mr->c;
  {
    ProfScope ps(c, KF_MR_PROLONG);
    const size_t NXY = (size_t)c->g.nx * c->g.ny, n = NXY * c->g.nz;
    k_mr_lerp<<<dim3(c->num_sms * 8, 3), 256, 0, c->stream>>>(n, NXY, theta, u0, v0, w0, u1, v1, w1,
                                                             mr->ul, mr->vl, mr->wl);
    c->launches++;
  }
  return prolong(mr, mr->ul, mr->vl, mr->wl, uf, vf, wf);
}

cudaError_t restrict_T(afid_mr* mr, const double* Tf, double* Tc) {
  afid_ctx* c = mr->c;
  ProfScope ps(c, KF_MR_RESTRICT);
  k_mr_restrict<<<c->num_sms * 8, 256, 0, c->stream>>>(c->g, mr->gf, mr->r[0], mr->r[1], mr->r[2], Tf, Tc);
  c->launches++;
  return cudaGetLastError();
}

// one refined substep l of size dts with the fine velocity in uf, vf, wf
cudaError_t scalar_substep(afid_mr* mr, int l, double dts, double* Tf) {
  afid_ctx* c = mr->c;
  const Grid& gf = mr->gf;
  {
    ProfScope ps(c, KF_CNTAB);
    if (cn_tables_grid(gf, mr->mf, l, dts, mr->scal, c->phys.nu, c->phys.kappa, mr->cntab, c->stream))
      return cudaGetLastError();
    c->launches++;
  }
  {
    ProfScope ps(c, KF_MR_RHS);
    // shared-flux kernel when the blocks tile the plane exactly (no thread
    // leaves before the per-level barrier), the plain one otherwise
    const int wpr = gf.nx % 64 == 0 ? 2 : (gf.nx % 32 == 0 ? 1 : 0);
    const int by = wpr == 2 ? 4 : 8;
    const bool shared = wpr > 0 && gf.ny % by == 0;
    const int bx = shared ? 32 * wpr : 32;
    dim3 blk(bx, by);
    const long long bpp = (long long)ceil_div(gf.nx, bx) * ceil_div(gf.ny, by);
    const int kc = z_chunk(c, bpp, gf.nz);
    dim3 grd(ceil_div(gf.nx, bx), ceil_div(gf.ny, by), ceil_div(gf.nz, kc));
    const double ka = c->phys.kappa;
    const ScalarW sw{0.5 * gf.rdx, 0.5 * gf.rdy, ka * gf.rdx2, ka * gf.rdy2, 2.0 * (ka * gf.rdx2 + ka * gf.rdy2)};
    if (shared && wpr == 2)
      k_mr_scalar_rhs_sh<4, 2><<<grd, blk, 0, c->stream>>>(gf, mr->mf, sw, l, dts, mr->uf, mr->vf,
                                                           mr->wf, Tf, mr->HT, mr->RT, mr->cntab, kc);
    else if (shared)
      k_mr_scalar_rhs_sh<8, 1><<<grd, blk, 0, c->stream>>>(gf, mr->mf, sw, l, dts, mr->uf, mr->vf,
                                                           mr->wf, Tf, mr->HT, mr->RT, mr->cntab, kc);
    else
      k_mr_scalar_rhs<<<grd, blk, 0, c->stream>>>(gf, mr->mf, sw, l, dts, mr->uf, mr->vf, mr->wf,
                                                  Tf, mr->HT, mr->RT, mr->cntab, kc);
    c->launches++;
  }
  {
    ProfScope ps(c, KF_CN);
    cudaError_t e = cn_sweep_scalar(gf, mr->cntab, mr->RT, Tf, c->stream);
    if (e) return e;
    c->launches++;
  }
  return cudaGetLastError();
}

cudaError_t scalar_advance(afid_mr* mr, double dt, int n_sub, const double* u0, const double* v0,
                           const double* w0, const double* u1, const double* v1, const double* w1,
                           double* Tf) {
  const double start[3] = {0.0, rk_alpha(0), rk_alpha(0) + rk_alpha(1)};
  const double dts = dt / n_sub;
  for (int s = 0; s < n_sub; ++s) {
    for (int l = 0; l < 3; ++l) {
      const double theta = (s + start[l]) / n_sub;
      cudaError_t e = velocity_at(mr, theta, u0, v0, w0, u1, v1, w1, mr->uf, mr->vf, mr->wf);
      if (e) return e;
      e = scalar_substep(mr, l, dts, Tf);
      if (e) return e;
    }
  }
  return cudaSuccess;
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

afid_status check(std::initializer_list<const void*> ps) {
  for (const void* p : ps) {
    if (!p) return AFID_ERR_INVALID_ARG;
    if (!aligned16(p)) return AFID_ERR_ALIGNMENT;
  }
  return AFID_OK;
}

// lower index and upper weight of piecewise-linear interpolation from the
// increasing positions xc to x (clamped to the first / last interval)
void bracket(const std::vector<double>& xc, double x, int& a, double& t) {
  const int n = (int)xc.size();
  a = (int)(std::upper_bound(xc.begin(), xc.end(), x) - xc.begin()) - 1;
  a = std::max(0, std::min(a, n - 2));
  t = (x - xc[a]) / (xc[a + 1] - xc[a]);
}

// periodic table: coarse samples at (i + o) h, fine positions (I + o) h / r,
// o = 1/2 (centres) or 0 (faces): position in coarse index units
// (2I + 1 - r) / (2r) for centres, I / r for faces
void periodic_table(int n, int r, bool centred, int* idx, double* wt) {
  for (int I = 0; I < r * n; ++I) {
    const long long num = centred ? 2LL * I + 1 - r : (long long)I;
    const long long den = centred ? 2LL * r : (long long)r;
    long long q = num / den;
    if (num < 0 && q * den != num) q -= 1;  // floor
    const long long rem = num - q * den;
    idx[I] = (int)(((q % n) + n) % n);
    wt[I] = (double)rem / (double)den;
  }
}

void free_mr(afid_mr* mr) {
  void* ps[] = {mr->metric_buf, mr->itab, mr->wtab, mr->cntab, mr->scal, mr->uf, mr->vf, mr->wf, mr->HT,
                mr->RT, mr->u0, mr->v0, mr->w0, mr->ul, mr->vl, mr->wl, mr->Tc, mr->stat_buf};
  for (void* p : ps)
    if (p) cudaFree(p);
}

}  // namespace
}  // namespace afid

extern "C" {

afid_status afid_mr_create(afid_ctx* c, int rx, int ry, int rz, afid_mr** out) {
  if (!out) return AFID_ERR_INVALID_ARG;
  *out = nullptr;
  if (!c || (c->flags & AFID_POISSON_ONLY) || !c->zf_host) return AFID_ERR_INVALID_ARG;
  if (rx < 1 || ry < 1 || rz < 1 || rx > 8 || ry > 8 || rz > 8) return AFID_ERR_INVALID_ARG;
  const Grid& g = c->g;
  const long long nxf = (long long)rx * g.nx, nyf = (long long)ry * g.ny, nzf = (long long)rz * g.nz;
  if (nxf > 32768 || nyf > 32768 || nzf > 32768) return AFID_ERR_UNSUPPORTED_SIZE;
  afid_mr* mr = new (std::nothrow) afid_mr;
  if (!mr) return AFID_ERR_OOM;
  std::memset(mr, 0, sizeof(*mr));
  mr->c = c;
  mr->r[0] = rx;
  mr->r[1] = ry;
  mr->r[2] = rz;
  Grid& gf = mr->gf;
  gf.nx = (int)nxf;
  gf.ny = (int)nyf;
  gf.nz = (int)nzf;
  gf.dx = c->lx / gf.nx;
  gf.dy = c->ly / gf.ny;
  gf.rdx = 1.0 / gf.dx;
  gf.rdy = 1.0 / gf.dy;
  gf.rdx2 = gf.rdx * gf.rdx;
  gf.rdy2 = gf.rdy * gf.rdy;

  // fine faces nesting the coarse ones
  const int nz = g.nz;
  const double* zf = c->zf_host;
  std::vector<double> zff((size_t)gf.nz + 1);
  afid_mr_faces(mr, zff.data());
  std::vector<double> flat;
  std::vector<size_t> offs;
  metric_host(gf.nz, gf.rdx2, gf.rdy2, zff.data(), flat, offs);

  // prolongation tables
  const size_t len[T_COUNT] = {(size_t)gf.nx, (size_t)gf.nx, (size_t)gf.ny, (size_t)gf.ny,
                               (size_t)gf.nz, (size_t)gf.nz + 1};
  size_t tot = 0;
  for (int t = 0; t < T_COUNT; ++t) {
    mr->off[t] = tot;
    tot += len[t];
  }
  std::vector<int> it(tot);
  std::vector<double> wt(tot);
  periodic_table(g.nx, rx, false, it.data() + mr->off[T_XF], wt.data() + mr->off[T_XF]);
  periodic_table(g.nx, rx, true, it.data() + mr->off[T_XC], wt.data() + mr->off[T_XC]);
  periodic_table(g.ny, ry, false, it.data() + mr->off[T_YF], wt.data() + mr->off[T_YF]);
  periodic_table(g.ny, ry, true, it.data() + mr->off[T_YC], wt.data() + mr->off[T_YC]);
  std::vector<double> zext((size_t)nz + 2), zfc(zf, zf + nz + 1);
  zext[0] = zf[0];
  for (int k = 0; k < nz; ++k) zext[(size_t)k + 1] = 0.5 * (zf[k] + zf[k + 1]);
  zext[(size_t)nz + 1] = zf[nz];
  for (int K = 0; K < gf.nz; ++K)
    bracket(zext, 0.5 * (zff[K] + zff[(size_t)K + 1]), it[mr->off[T_ZC] + K], wt[mr->off[T_ZC] + K]);
  for (int K = 0; K <= gf.nz; ++K)
    bracket(zfc, zff[K], it[mr->off[T_ZF] + K], wt[mr->off[T_ZF] + K]);

  // device buffers
  bool ok = true;
  auto get = [&](size_t count) -> double* {
    if (!ok) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(double)) != cudaSuccess) {
      ok = false;
      cudaGetLastError();
      return nullptr;
    }
    mr->bytes += count * sizeof(double);
    return static_cast<double*>(p);
  };
  const size_t NXYf = (size_t)gf.nx * gf.ny, NXY = (size_t)g.nx * g.ny;
  const size_t ncf = NXYf * gf.nz, nff = NXYf * (gf.nz + 1), nc = NXY * nz, nf = NXY * (nz + 1);
  mr->metric_buf = get(flat.size());
  mr->wtab = get(tot);
  if (ok && cudaMalloc(reinterpret_cast<void**>(&mr->itab), tot * sizeof(int)) != cudaSuccess) {
    ok = false;
    cudaGetLastError();
  }
  mr->cntab = get((size_t)3 * CN_TAB_ARRAYS * (gf.nz + 1));
  mr->scal = get(S_COUNT);
  mr->uf = get(ncf);
  mr->vf = get(ncf);
  mr->wf = get(nff);
  mr->HT = get(nff);
  mr->RT = get(nff);
  mr->u0 = get(nc);
  mr->v0 = get(nc);
  mr->w0 = get(nf);
  mr->ul = get(nc);
  mr->vl = get(nc);
  mr->wl = get(nf);
  mr->Tc = get(nf);
  mr->stat_buf = get((size_t)(gf.nz + 1) * AFID_STAT_NQ + 8);
  if (ok) {
    ok = cudaMemcpy(mr->metric_buf, flat.data(), flat.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(mr->itab, it.data(), tot * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(mr->wtab, wt.data(), tot * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(mr->cntab, 0, (size_t)3 * CN_TAB_ARRAYS * (gf.nz + 1) * sizeof(double)) == cudaSuccess &&
         cudaMemset(mr->scal, 0, S_COUNT * sizeof(double)) == cudaSuccess &&
         cudaMemset(mr->HT, 0, nff * sizeof(double)) == cudaSuccess &&
         cudaMemset(mr->RT, 0, nff * sizeof(double)) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_mr(mr);
    delete mr;
    return AFID_ERR_OOM;
  }
  mr->mf = metric_view(static_cast<const double*>(mr->metric_buf), offs);
  *out = mr;
  return AFID_OK;
}

afid_status afid_mr_destroy(afid_mr* mr) {
  if (!mr) return AFID_ERR_INVALID_ARG;
  cudaStreamSynchronize(mr->c->stream);
  free_mr(mr);
  delete mr;
  return AFID_OK;
}

afid_status afid_mr_dims(const afid_mr* mr, int* nxf, int* nyf, int* nzf) {
  if (!mr || !nxf || !nyf || !nzf) return AFID_ERR_INVALID_ARG;
  *nxf = mr->gf.nx;
  *nyf = mr->gf.ny;
  *nzf = mr->gf.nz;
  return AFID_OK;
}

size_t afid_mr_workspace_bytes(const afid_mr* mr) { return mr ? mr->bytes : 0; }

afid_status afid_mr_faces(const afid_mr* mr, double* zf_out) {
  if (!mr || !zf_out) return AFID_ERR_INVALID_ARG;
  const int nz = mr->c->g.nz, rz = mr->r[2];
  const double* zf = mr->c->zf_host;
  for (int k = 0; k < nz; ++k)
    for (int m = 0; m < rz; ++m) zf_out[(size_t)k * rz + m] = zf[k] + (zf[k + 1] - zf[k]) * m / rz;
  zf_out[(size_t)nz * rz] = zf[nz];
  return AFID_OK;
}

afid_status afid_mr_prolong(afid_mr* mr, const double* u0, const double* v0, const double* w0,
                            const double* u1, const double* v1, const double* w1, double theta,
                            double* uf, double* vf, double* wf) {
  if (!mr || !std::isfinite(theta) || theta < 0.0 || theta > 1.0) return AFID_ERR_INVALID_ARG;
  afid_status st = check({u0, v0, w0, uf, vf, wf});
  if (st) return st;
  if (theta != 0.0 && (st = check({u1, v1, w1}))) return st;
  return velocity_at(mr, theta, u0, v0, w0, u1, v1, w1, uf, vf, wf) ? AFID_ERR_CUDA : AFID_OK;
}

afid_status afid_mr_restrict(afid_mr* mr, const double* Tf, double* Tc) {
  if (!mr) return AFID_ERR_INVALID_ARG;
  afid_status st = check({Tf, Tc});
  if (st) return st;
  return restrict_T(mr, Tf, Tc) ? AFID_ERR_CUDA : AFID_OK;
}

afid_status afid_mr_scalar_advance(afid_mr* mr, double dt, int n_sub, const double* u0,
                                   const double* v0, const double* w0, const double* u1,
                                   const double* v1, const double* w1, double* Tf) {
  if (!mr || !(dt > 0.0) || !std::isfinite(dt) || n_sub < 1) return AFID_ERR_INVALID_ARG;
  afid_status st = check({u0, v0, w0, u1, v1, w1, Tf});
  if (st) return st;
  return scalar_advance(mr, dt, n_sub, u0, v0, w0, u1, v1, w1, Tf) ? AFID_ERR_CUDA : AFID_OK;
}

afid_status afid_mr_statistics(afid_mr* mr, const double* u, const double* v, const double* w,
                               const double* Tf, double* profiles, afid_stats* out) {
  if (!mr) return AFID_ERR_INVALID_ARG;
  afid_status st = check({u, v, w, Tf});
  if (st) return st;
  afid_ctx* c = mr->c;
  const Grid& gf = mr->gf;
  if (prolong(mr, u, v, w, mr->uf, mr->vf, mr->wf)) return AFID_ERR_CUDA;
  if (statistics_grid(gf, mr->mf, c->phys, mr->uf, mr->vf, mr->wf, Tf, mr->stat_buf, c->stream))
    return AFID_ERR_CUDA;
  c->launches += 2;
  const size_t np = (size_t)(gf.nz + 1) * AFID_STAT_NQ;
  double sc[8];
  if (profiles &&
      cudaMemcpyAsync(profiles, mr->stat_buf, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream))
    return AFID_ERR_CUDA;
  if (cudaMemcpyAsync(sc, mr->stat_buf + np, sizeof(sc), cudaMemcpyDeviceToHost, c->stream))
    return AFID_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream)) return AFID_ERR_CUDA;
  if (out) {
    out->nu_volume = sc[0];
    out->nu_bottom = sc[1];
    out->nu_top = sc[2];
    out->tau_bottom = sc[3];
    out->tau_top = sc[4];
    out->re_tau = sc[5];
    out->ke = sc[6];
  }
  return AFID_OK;
}

afid_status afid_mr_step(afid_mr* mr, double dt, int n_sub, double* u, double* v, double* w, double* p,
                         double* Hu, double* Hv, double* Hw, double* Tf, afid_info* info) {
  if (!mr || !(dt > 0.0) || !std::isfinite(dt) || n_sub < 1) return AFID_ERR_INVALID_ARG;
  afid_status st = check({u, v, w, p, Hu, Hv, Hw, Tf});
  if (st) return st;
  afid_ctx* c = mr->c;
  const size_t NXY = (size_t)c->g.nx * c->g.ny, nc = NXY * c->g.nz, nf = NXY * (c->g.nz + 1);
  if (cudaMemcpyAsync(mr->u0, u, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) ||
      cudaMemcpyAsync(mr->v0, v, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) ||
      cudaMemcpyAsync(mr->w0, w, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream))
    return AFID_ERR_CUDA;
  if (restrict_T(mr, Tf, mr->Tc)) return AFID_ERR_CUDA;
  for (int l = 0; l < 3; ++l) {
    st = afid_rk3_substep(c, l, dt, u, v, w, mr->Tc, p, Hu, Hv, Hw, nullptr, l == 2 ? info : nullptr);
    if (st != AFID_OK && st != AFID_ERR_NOT_CONVERGED && st != AFID_ERR_INCONSISTENT_RHS) return st;
  }
  if (scalar_advance(mr, dt, n_sub, mr->u0, mr->v0, mr->w0, u, v, w, Tf)) return AFID_ERR_CUDA;
  return st;
}

}  // extern "C"
