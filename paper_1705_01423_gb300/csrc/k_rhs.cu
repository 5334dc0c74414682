// Explicit terms H and Crank-Nicolson right-hand sides R of one RK3 substep
// (Sec. 2.1), z-marching formulation.
//
// On this part FP64 issues at 2 instructions per clock per SM, 1/64 of FP32,
// so the kernel is bound by the number of FP64 instructions per grid point,
// not by HBM. The conservative advection operator is a difference of face
// fluxes; here every face flux is computed once and shared:
//   * z: each thread owns one (x, y) column and walks k upwards, carrying the
//     flux through face k+1 (cell k for w, T) to the next step in registers;
//   * x: a warp spans 32 consecutive x; the neighbour's flux comes by shuffle,
//     across the two warps of a 64-wide block row through shared memory;
//   * y: the block spans BY rows; fluxes of the neighbouring row come through a
//     double-buffered shared-memory exchange (one barrier per k).
// Only the block's outer edges recompute a neighbour's flux (every lane of
// the edge warp issues that code, since masked lanes cost the same issue
// slots), so wider blocks spend fewer operations on edges. The fluxes of u
// through its x faces and of v through its y faces need no exchange at all:
// their difference (u_i + u_i+1)^2 - (u_i-1 + u_i)^2 is formed as
// (u_i+1 - u_i-1)(u_i+1 + u_i-1 + 2 u_i), whose sum the horizontal diffusion
// needs anyway (the same operation count, and more accurate where the two
// squares nearly cancel).
// Constant factors (1/2, 1/4, 1/dx, dt gamma_l, ...) are folded; the
// wall-normal term alpha_l dt d dzz q of R takes its three coefficients per
// row from the substep's Crank-Nicolson table. The z-march of a column is
// split into chunks (blockIdx.z) so that the grid balances over the SMs; a
// chunk starts from the fluxes of the plane below it.
// Same discretisation as the point-wise formulation it replaces:
//   u: [(u_i+u_i+1)^2 - (u_i-1+u_i)^2]/(4dx) + [C_i,j+1 - C_i,j]/(4dy)
//      + [Fz_k+1 - Fz_k]/(4 dzc_k), C_i,j = (v_i-1,j + v_i,j)(u_i,j-1 + u_i,j),
//      Fz_k = (w_i-1,k + w_i,k)(u_k-1 + u_k) (zero on the walls);
//   v: symmetric; w, T on face k: x/y fluxes uf (q_i-1 + q_i) with
//      uf = (dzc_k-1 u_k-1 + dzc_k u_k)/(2 dzf_k), z fluxes at cell centres
//      (w_k + w_k+1)(q_k + q_k+1)/4.
#include "afid_internal.cuh"

namespace afid {

// Scalar factors of the kernel, formed on the host: as kernel parameters they
// sit in the constant bank, where an FMA reads them directly (computed in the
// kernel they would hold registers or be recomputed in the loop).
struct PhysR {
  double buoy, ubot, utop;
  double qx, qy;          // 1/4 of the inverse spacings
  double hx, hy;          // 1/2 of the inverse spacings
  double nrx, nry, nl0;   // nu / dx^2, nu / dy^2, 2 nu (1/dx^2 + 1/dy^2)
  double krx, kry, kl0;   // the same with kappa
};

// WPR warps per block row: 1 (BX = min(32, nx), BY = 8; two blocks per SM) or
// 2 (BX = 64, BY = 8, one 512-thread block per SM; the two warps of a row pass
// their facing edge fluxes through shared memory, so only the block's outer
// edges recompute neighbour fluxes, and 8 rows put the y edge on 1/8 of them).
// TM: 0 no temperature, 1 temperature advanced (HT, RT written), 2 T only
// supplies the buoyancy of the w equation (T kept on another grid).
template <int TM, int BY, int WPR>
__global__ void __launch_bounds__(32 * WPR * BY, WPR * BY >= 16 ? 1 : 2) k_rhs_zm(Grid g, Metric m, PhysR ph, int l, double dt_in,
                                                    const double* __restrict__ scal,
                                                    const double* __restrict__ u,
                                                    const double* __restrict__ v,
                                                    const double* __restrict__ w,
                                                    const double* __restrict__ T,
                                                    const double* __restrict__ p,
                                                    double* __restrict__ Hu, double* __restrict__ Hv,
                                                    double* __restrict__ Hw, double* __restrict__ HT,
                                                    double* __restrict__ Ru, double* __restrict__ Rv,
                                                    double* __restrict__ Rw, double* __restrict__ RT,
                                                    const double* __restrict__ cnt, int kchunk) {
  constexpr bool HAS_T = TM == 1, BUOY = TM != 0;
  const int BX = blockDim.x;  // min(32, nx) or 64
  const int SW = WPR == 1 ? BX : 32;  // shuffle width: one block row per warp segment
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * BX + tx, j = blockIdx.y * BY + ty;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ip = wrap_next(i, nx), im = wrap_prev(i, nx);
  const int jp = wrap_next(j, ny), jm = wrap_prev(j, ny);
  const size_t NXY = (size_t)nx * ny;
  const bool last_lane = tx == BX - 1, last_row = ty == BY - 1;

  // The right-hand sides are written multiplied by the reciprocal pivot m_k of
  // their Crank-Nicolson row (the sweep's forward elimination then needs no
  // multiply): every coefficient of R -- dt gamma_l, dt rho_l, the
  // alpha_l dt d dzz weights of q_{k-1}, q_{k+1}, q_k and the pressure-gradient
  // factors -- comes pre-scaled per plane from the substep's table (k_cn_tables,
  // cells / faces (nu) / faces (kappa); read as cnt[(set * CN_TAB_ARRAYS + a) * L
  // + k], one base pointer keeping the register count down). dt itself enters
  // only through those tables.
  (void)dt_in;
  (void)scal;
  const int L = nz + 1;
  // this block's range of k (the z-march is split into chunks for load balance)
  const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
  // horizontal diffusion nu (d_xx + d_yy) q as nu rdx2 (q_i+1 + q_i-1) +
  // nu rdy2 (q_j+1 + q_j-1) - 2 nu (rdx2 + rdy2) q: the diffusivity folded
  // into the three weights (kappa for T)
  const double qx = ph.qx, qy = ph.qy, hx = ph.hx, hy = ph.hy;
  const double nrx = ph.nrx, nry = ph.nry, nl0 = ph.nl0, krx = ph.krx, kry = ph.kry, kl0 = ph.kl0;

  // shared y-exchange: [buffer][quantity][row][x] (C, fyw, fyt); x-edge
  // exchange between the two warps of a row: fxw, fxt of x = 32
  __shared__ double sx[2][3][BY][32 * WPR];
  __shared__ double sxe[2][2][BY];

  const size_t col = (size_t)j * nx + i;
  const size_t cim = (size_t)j * nx + im, cip = (size_t)j * nx + ip;
  const size_t cjm = (size_t)jm * nx + i, cjp = (size_t)jp * nx + i;
  const size_t cjpim = (size_t)jp * nx + im, cjmip = (size_t)jm * nx + ip;

  // column values carried along k (state at k = k0)
  const size_t c0 = (size_t)k0 * NXY;
  double u0 = u[c0 + col], v0 = v[c0 + col];
  double w0 = w[c0 + col], wk1 = w[c0 + NXY + col];
  double t0 = BUOY ? T[c0 + col] : 0.0, tk1 = BUOY ? T[c0 + NXY + col] : 0.0;
  double wim0 = w[c0 + cim], wjm0 = w[c0 + cjm];  // face k at (i-1), (j-1)
  double fzu = 0.0, fzv = 0.0;          // u, v z-fluxes through face k (wall: 0)
  double fzw = 0.0, fzt = 0.0;          // w, T z-fluxes at cell k-1
  double ukm = ph.ubot, vkm = 0.0;      // u, v at k-1 (wall values at k = 0)
  double uipkm = 0.0, vjpkm = 0.0;      // u(i+1), v(j+1) at k-1
  double wkm = 0.0, tkm = 0.0, pkm = 0.0;
  if (k0 > 0) {  // interior chunk start: the same quantities from plane k0 - 1
    const size_t cm = c0 - NXY;
    ukm = u[cm + col];
    vkm = v[cm + col];
    uipkm = u[cm + cip];
    vjpkm = v[cm + cjp];
    wkm = w[cm + col];
    tkm = HAS_T ? T[cm + col] : 0.0;
    pkm = p[cm + col];
    fzu = (wim0 + w0) * (ukm + u0);
    fzv = (wjm0 + w0) * (vkm + v0);
    const double ws = wkm + w0;
    fzw = ws * ws;
    fzt = HAS_T ? ws * (tkm + t0) : 0.0;
  }

  for (int k = k0; k < k1; ++k) {
    const size_t c = (size_t)k * NXY;
    const int buf = k & 1;
    // ---------------------------------------------------------------- loads at plane k
    const double uip = u[c + cip], uim = u[c + cim], ujp = u[c + cjp], ujm = u[c + cjm];
    const double vip = v[c + cip], vim = v[c + cim], vjp = v[c + cjp], vjm = v[c + cjm];
    const double ukp = k < nz - 1 ? u[c + NXY + col] : ph.utop;
    const double vkp = k < nz - 1 ? v[c + NXY + col] : 0.0;
    const double wk1im = w[c + NXY + cim], wk1jm = w[c + NXY + cjm];
    const double p0 = p[c + col];

    // ---------------------------------------------------------------- shared fluxes (cell k)
    const double C = (vim + v0) * (ujm + u0);        // corner (x-face i, y-face j), x4
    const double fzu1 = k < nz - 1 ? (wk1im + wk1) * (u0 + ukp) : 0.0;  // face k+1, x4
    const double fzv1 = k < nz - 1 ? (wk1jm + wk1) * (v0 + vkp) : 0.0;
    const double wsum = w0 + wk1;                     // 2 w at cell centre k
    const double fzw1 = wsum * wsum;                  // cell k, x4
    const double fzt1 = HAS_T ? wsum * (t0 + tk1) : 0.0;

    // face-k quantities (k >= 1): uf, vf and the x/y fluxes of w and T
    double ufi = 0.0, vfj = 0.0, fxw = 0.0, fyw = 0.0, fxt = 0.0, fyt = 0.0;
    double wip = 0.0, wjp = 0.0, tip = 0.0, tim = 0.0, tjp = 0.0, tjm = 0.0;
    if (k > 0) {
      const double wlo = m.wlo[k], whi = m.whi[k];
      ufi = fma(wlo, ukm, whi * u0);
      vfj = fma(wlo, vkm, whi * v0);
      wip = w[c + cip];
      wjp = w[c + cjp];
      fxw = ufi * (wim0 + w0);                        // x-face i, x2
      fyw = vfj * (wjm0 + w0);                        // y-face j, x2
      if (HAS_T) {
        tip = T[c + cip];
        tim = T[c + cim];
        tjp = T[c + cjp];
        tjm = T[c + cjm];
        fxt = ufi * (tim + t0);
        fyt = vfj * (tjm + t0);
      }
    }
    // ---------------------------------------------------------------- exchange
    sx[buf][0][ty][tx] = C;
    sx[buf][1][ty][tx] = fyw;
    sx[buf][2][ty][tx] = fyt;
    if (WPR == 2 && tx == 32) {
      sxe[buf][0][ty] = fxw;
      sxe[buf][1][ty] = fxt;
    }
    __syncthreads();
    // x neighbours by shuffle (lane i+1 / i-1 of the same row)
    const unsigned FULL = 0xffffffffu;
    double Cip = __shfl_down_sync(FULL, C, 1, SW);
    double fxw1 = __shfl_down_sync(FULL, fxw, 1, SW);
    double fxt1 = __shfl_down_sync(FULL, fxt, 1, SW);
    if (WPR == 2 && tx == 31) {  // facing edges of the two warps of a row
      Cip = sx[buf][0][ty][32];
      fxw1 = sxe[buf][0][ty];
      fxt1 = sxe[buf][1][ty];
    }
    // Block-edge lanes recompute the neighbour's fluxes. The warp-uniform
    // vote keeps these blocks a real branch taken only by the warps that
    // hold an edge lane (if-converted, every warp would issue them).
    if (__any_sync(FULL, last_lane)) {
      if (last_lane) {
        Cip = (v0 + vip) * (u[c + cjmip] + uip);
        if (k > 0) {
          const double ufip = fma(m.wlo[k], uipkm, m.whi[k] * uip);
          fxw1 = ufip * (w0 + wip);
          if (HAS_T) fxt1 = ufip * (t0 + tip);
        }
      }
    }
    // y neighbours from shared memory (rows j+1 / j-1 of the block)
    const int typ = last_row ? ty : ty + 1;
    double Cjp = sx[buf][0][typ][tx];
    double fyw1 = sx[buf][1][typ][tx];
    double fyt1 = sx[buf][2][typ][tx];
    if (__any_sync(FULL, last_row)) {
      if (last_row) {
        Cjp = (v[c + cjpim] + vjp) * (u0 + ujp);
        fyw1 = 0.0;
        fyt1 = 0.0;
        if (k > 0) {
          const double vfjp = fma(m.wlo[k], vjpkm, m.whi[k] * vjp);
          fyw1 = vfjp * (w0 + wjp);
          if (HAS_T) fyt1 = vfjp * (t0 + tjp);
        }
      }
    }

    // ---------------------------------------------------------------- u, v at cell k
    const double qz = cnt[CN_QZ * L + k];  // dzc^-1 / 4
    {
      // x flux difference (u_i + u_i+1)^2 - (u_i-1 + u_i)^2 as
      // (u_i+1 - u_i-1)(u_i+1 + u_i-1 + 2 u_i), its sum shared with the diffusion:
      // no neighbour's flux needed
      const double sxu = uip + uim;
      const double dfx = (uip - uim) * fma(2.0, u0, sxu);
      const double A = fma(fzu1 - fzu, qz, fma(Cjp - C, qy, dfx * qx));
      const double H = fma(nrx, sxu, fma(nry, ujp + ujm, fma(-nl0, u0, -A)));
      const double z = fma(cnt[CN_MEA * L + k], ukm, fma(cnt[CN_MEC * L + k], ukp, fma(cnt[CN_MED * L + k], u0, -cnt[CN_MGX * L + k] * (p0 - p[c + cim]))));
      double r = fma(cnt[CN_MCG * L + k], H, z);
      if (l > 0) r = fma(cnt[CN_MCR * L + k], Hu[c + col], r);
      Hu[c + col] = H;
      Ru[c + col] = r;
    }
    {
      const double syv = vjp + vjm;  // y flux difference of v, as for u in x
      const double dfy = (vjp - vjm) * fma(2.0, v0, syv);
      const double A = fma(fzv1 - fzv, qz, fma(dfy, qy, (Cip - C) * qx));
      const double H = fma(nrx, vip + vim, fma(nry, syv, fma(-nl0, v0, -A)));
      const double z = fma(cnt[CN_MEA * L + k], vkm, fma(cnt[CN_MEC * L + k], vkp, fma(cnt[CN_MED * L + k], v0, -cnt[CN_MGY * L + k] * (p0 - p[c + cjm]))));
      double r = fma(cnt[CN_MCG * L + k], H, z);
      if (l > 0) r = fma(cnt[CN_MCR * L + k], Hv[c + col], r);
      Hv[c + col] = H;
      Rv[c + col] = r;
    }
    // ---------------------------------------------------------------- w, T on face k
    if (k == 0) {
      Hw[col] = 0.0;
      Hw[(size_t)nz * NXY + col] = 0.0;
      if (HAS_T) {
        HT[col] = 0.0;
        HT[(size_t)nz * NXY + col] = 0.0;
      }
    } else {
      const double qzf = cnt[CN_QZF * L + k];  // dzf^-1 / 4
      {
        const double A = fma(fzw1 - fzw, qzf, fma(fyw1 - fyw, hy, (fxw1 - fxw) * hx));
        double H = fma(nrx, wip + wim0, fma(nry, wjp + wjm0, fma(-nl0, w0, -A)));
        if (BUOY) H = fma(ph.buoy, t0, H);
        const double z = fma(cnt[(CN_TAB_ARRAYS + CN_MEA) * L + k], wkm, fma(cnt[(CN_TAB_ARRAYS + CN_MEC) * L + k], wk1, fma(cnt[(CN_TAB_ARRAYS + CN_MED) * L + k], w0, -cnt[(CN_TAB_ARRAYS + CN_MGX) * L + k] * (p0 - pkm))));
        double r = fma(cnt[(CN_TAB_ARRAYS + CN_MCG) * L + k], H, z);
        if (l > 0) r = fma(cnt[(CN_TAB_ARRAYS + CN_MCR) * L + k], Hw[c + col], r);
        Hw[c + col] = H;
        Rw[c + col] = r;
      }
      if (HAS_T) {
        const double A = fma(fzt1 - fzt, qzf, fma(fyt1 - fyt, hy, (fxt1 - fxt) * hx));
        const double H = fma(krx, tip + tim, fma(kry, tjp + tjm, fma(-kl0, t0, -A)));
        const double z = fma(cnt[(2 * CN_TAB_ARRAYS + CN_MEA) * L + k], tkm, fma(cnt[(2 * CN_TAB_ARRAYS + CN_MEC) * L + k], tk1, cnt[(2 * CN_TAB_ARRAYS + CN_MED) * L + k] * t0));
        double r = fma(cnt[(2 * CN_TAB_ARRAYS + CN_MCG) * L + k], H, z);
        if (l > 0) r = fma(cnt[(2 * CN_TAB_ARRAYS + CN_MCR) * L + k], HT[c + col], r);
        HT[c + col] = H;
        RT[c + col] = r;
      }
    }
    // ---------------------------------------------------------------- carry to k+1
    fzu = fzu1;
    fzv = fzv1;
    fzw = fzw1;
    fzt = fzt1;
    ukm = u0;
    vkm = v0;
    uipkm = uip;
    vjpkm = vjp;
    wkm = w0;
    tkm = t0;
    pkm = p0;
    if (k < nz - 1) {
      u0 = ukp;
      v0 = vkp;
      w0 = wk1;
      t0 = tk1;
      wim0 = wk1im;
      wjm0 = wk1jm;
      wk1 = w[c + 2 * NXY + col];
      if (BUOY) tk1 = T[c + 2 * NXY + col];
    }
  }
}

cudaError_t rk3_explicit(afid_ctx* c, int l, double dt, const double* u, const double* v,
                         const double* w, const double* T, const double* p, double* Hu,
                         double* Hv, double* Hw, double* HT) {
  ProfScope ps(c, KF_RHS);
  const Grid& g = c->g;
  const bool wide = g.nx % 64 == 0;
  const int BY = 8;
  const int bx = wide ? 64 : x_block(g.nx, 32);
  // split the z-march into chunks so that the grid is about eight waves of
  // two resident blocks per SM (the chunk start re-reads one plane)
  const long long bxy = (long long)(g.nx / bx) * (g.ny / BY);
  const long long want = 16LL * c->num_sms;
  int nch = (int)((want + bxy - 1) / bxy);
  nch = nch < 1 ? 1 : nch;
  const int max_ch = g.nz / 16 > 0 ? g.nz / 16 : 1;
  nch = nch > max_ch ? max_ch : nch;
  const int kchunk = (g.nz + nch - 1) / nch;
  nch = (g.nz + kchunk - 1) / kchunk;
  dim3 blk(bx, BY), grd(g.nx / bx, g.ny / BY, nch);
  const double nu = c->phys.nu, ka = c->phys.kappa;
  PhysR ph{c->phys.buoyancy, c->phys.u_bot, c->phys.u_top, 0.25 * g.rdx, 0.25 * g.rdy, 0.5 * g.rdx, 0.5 * g.rdy,
           nu * g.rdx2, nu * g.rdy2, 2.0 * (nu * g.rdx2 + nu * g.rdy2),
           ka * g.rdx2, ka * g.rdy2, 2.0 * (ka * g.rdx2 + ka * g.rdy2)};
#define AFID_RHS(HT_, BY_, W_)                                                                     \
  k_rhs_zm<HT_, BY_, W_><<<grd, blk, 0, c->stream>>>(g, c->m, ph, l, dt, c->scal, u, v, w, T, p, Hu, Hv, \
                                                     Hw, HT, c->R[0], c->R[1], c->R[2], c->R[3],         \
                                                     c->cntab, kchunk)
  if (T && HT) {
    if (wide) AFID_RHS(1, 8, 2);
    else AFID_RHS(1, 8, 1);
  } else if (T) {
    if (wide) AFID_RHS(2, 8, 2);
    else AFID_RHS(2, 8, 1);
  } else {
    if (wide) AFID_RHS(0, 8, 2);
    else AFID_RHS(0, 8, 1);
  }
#undef AFID_RHS
  c->launches++;
  return cudaGetLastError();
}

}  // namespace afid
