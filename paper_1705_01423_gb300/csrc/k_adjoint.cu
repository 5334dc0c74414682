// Hand-written adjoints (exact transposes) of the pressure correction and of
// one RK3 / Crank-Nicolson substep, with dt held constant.
//
// Poisson solve S (mean removal + L^-1 + gauge): L = W_c^-1 K with K
// symmetric, so S^T y = W_c S(W_c^-1 y), W_c the cell volumes.
// Projection (u, v, w, p) -> (u - s G phi, p + (I - beta dzz) phi),
// phi = S D u / s: with face weights W_f and h = W_f^-1 g_vel,
// q = W_c^-1 g_p, psi = S(s D h + q - beta dzz q), the transpose is
// g_vel <- W_f (h - G psi / s), g_p unchanged (D^T = -W_f G W_c^-1).
// Wall planes of w and T are boundary data, not unknowns: their cotangents
// are returned as zero.
#include "afid_internal.cuh"

namespace afid {

__device__ __forceinline__ size_t ix(const Grid& g, int k, int j, int i) {
  return ((size_t)k * g.ny + j) * g.nx + i;
}

static inline dim3 pgrid(const Grid& g, int& bx) {
  bx = x_block(g.nx, 128);
  return dim3(g.nx / bx, g.ny, g.nz);
}

// ---------------------------------------------------------------------------
// out = in * dzc_k (forward) or in / dzc_k
__global__ void k_scale_cells(Grid g, Metric m, const double* __restrict__ in,
                              double* __restrict__ out, int mul) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const size_t c = ix(g, k, j, i);
  out[c] = mul ? in[c] * m.dzc[k] : in[c] * m.rdzc[k];
}

cudaError_t scale_cells(afid_ctx* c, const double* in, double* out, bool mul) {
  ProfScope ps(c, KF_ADJ);
  int bx;
  dim3 grd = pgrid(c->g, bx);
  k_scale_cells<<<grd, bx, 0, c->stream>>>(c->g, c->m, in, out, mul ? 1 : 0);
  c->launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Projection adjoint, first half: rhs_psi = s D(h) + q - beta dzz q into `out`.
__global__ void k_adj_proj_pre(Grid g, Metric m, const double* __restrict__ gu,
                               const double* __restrict__ gv, const double* __restrict__ gw,
                               const double* __restrict__ gp, const double* __restrict__ scal,
                               double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const double s = scal[S_PROJ_S], beta = scal[S_PROJ_BETA];
  const int ip = wrap_next(i, g.nx), jp = wrap_next(j, g.ny);
  const size_t c = ix(g, k, j, i), NXY = (size_t)g.nx * g.ny;
  const double rA = 1.0 / (g.dx * g.dy);
  const double rc = rA * m.rdzc[k];
  const double hu0 = gu[c] * rc, hu1 = gu[ix(g, k, j, ip)] * rc;
  const double hv0 = gv[c] * rc, hv1 = gv[ix(g, k, jp, i)] * rc;
  const double hw0 = k > 0 ? gw[c] * rA * m.rdzf[k] : 0.0;
  const double hw1 = k < g.nz - 1 ? gw[c + NXY] * rA * m.rdzf[k + 1] : 0.0;
  const double Dh = (hu1 - hu0) * g.rdx + (hv1 - hv0) * g.rdy + (hw1 - hw0) * m.rdzc[k];
  const double q0 = gp[c] * rc;
  const double qm = k > 0 ? gp[c - NXY] * rA * m.rdzc[k - 1] : q0;
  const double qp = k < g.nz - 1 ? gp[c + NXY] * rA * m.rdzc[k + 1] : q0;
  const double dzz = m.pc[k] * (qp - q0) - m.pa[k] * (q0 - qm);
  out[c] = s * Dh + q0 - beta * dzz;
}

// second half: g_vel -= W_f G psi / s; wall planes of gw zeroed.
__global__ void k_adj_proj_post(Grid g, Metric m, double* __restrict__ gu, double* __restrict__ gv,
                                double* __restrict__ gw, const double* __restrict__ psi,
                                const double* __restrict__ scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const double rs = scal[S_PROJ_RS];
  const int im = wrap_prev(i, g.nx), jm = wrap_prev(j, g.ny);
  const size_t c = ix(g, k, j, i), NXY = (size_t)g.nx * g.ny;
  const double f = psi[c];
  gu[c] -= g.dy * m.dzc[k] * rs * (f - psi[ix(g, k, j, im)]);
  gv[c] -= g.dx * m.dzc[k] * rs * (f - psi[ix(g, k, jm, i)]);
  if (k > 0) gw[c] -= g.dx * g.dy * rs * (f - psi[c - NXY]);
  else gw[c] = 0.0;
  if (k == g.nz - 1) gw[c + NXY] = 0.0;
}

cudaError_t project_adjoint_pre(afid_ctx* c, double* gu, double* gv, double* gw, const double* gp,
                                double, double) {
  ProfScope ps(c, KF_ADJ);
  int bx;
  dim3 grd = pgrid(c->g, bx);
  k_adj_proj_pre<<<grd, bx, 0, c->stream>>>(c->g, c->m, gu, gv, gw, gp, c->scal, c->phi);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t project_adjoint_post(afid_ctx* c, double* gu, double* gv, double* gw, double*,
                                 const double* psi, double, double) {
  ProfScope ps(c, KF_ADJ);
  int bx;
  dim3 grd = pgrid(c->g, bx);
  k_adj_proj_post<<<grd, bx, 0, c->stream>>>(c->g, c->m, gu, gv, gw, psi, c->scal);
  c->launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Substep adjoint, pointwise parts. Z = gH + dt gamma R (in place in gH);
// afterwards gH = dt rho R (cotangent of Hprev). R holds A^-T g for each
// Crank-Nicolson operator; wall planes of the face arrays carry nothing.
__global__ void k_adj_z(Grid g, double* gH0, double* gH1, double* gH2, double* gH3,
                        const double* R0, const double* R1, const double* R2, const double* R3,
                        double coef, int final_pass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const size_t c = ix(g, k, j, i), NXY = (size_t)g.nx * g.ny;
  double* gH[4] = {gH0, gH1, gH2, gH3};
  const double* R[4] = {R0, R1, R2, R3};
  for (int q = 0; q < 4; ++q) {
    if (!gH[q]) continue;
    const bool face = q >= 2;
    if (face && k == 0) {
      gH[q][c] = 0.0;
      gH[q][c + (size_t)g.nz * NXY] = 0.0;
      continue;
    }
    gH[q][c] = final_pass ? coef * R[q][c] : gH[q][c] + coef * R[q][c];
  }
}

// Transposed linearised explicit terms plus the direct Crank-Nicolson-side
// terms, scattered with atomics from each output point (i, j, k) to the inputs
// its forward stencil reads:
//   g_q   += E_q^T Z + dt alpha nu dzz_q^T R_q
//   g_p   -= dt alpha sum_q G_q^T R_q
struct PhysA {
  double nu, kappa, buoy;
};

__device__ __forceinline__ void aadd(double* a, size_t c, double v) { atomicAdd(a + c, v); }

__global__ void __launch_bounds__(128) k_adj_explicit(Grid g, Metric m, PhysA ph, int l, double dt,
                                                      const double* __restrict__ u,
                                                      const double* __restrict__ v,
                                                      const double* __restrict__ w,
                                                      const double* __restrict__ T,
                                                      const double* __restrict__ Zu,
                                                      const double* __restrict__ Zv,
                                                      const double* __restrict__ Zw,
                                                      const double* __restrict__ ZT,
                                                      const double* __restrict__ Ru,
                                                      const double* __restrict__ Rv,
                                                      const double* __restrict__ Rw,
                                                      const double* __restrict__ RT, double* gu,
                                                      double* gv, double* gw, double* gT, double* gp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int ip = wrap_next(i, nx), im = wrap_prev(i, nx);
  const int jp = wrap_next(j, ny), jm = wrap_prev(j, ny);
  const size_t NXY = (size_t)nx * ny;
  const double da = dt * rk_alpha(l);
  const size_t c = ix(g, k, j, i);
  const size_t cim = ix(g, k, j, im), cip = ix(g, k, j, ip), cjm = ix(g, k, jm, i), cjp = ix(g, k, jp, i);
  const double rdx = g.rdx, rdy = g.rdy, rdzc = m.rdzc[k];
  const double hx = 0.5 * rdx, hy = 0.5 * rdy, hz = 0.5 * rdzc;

  // ------------------------------------------------------------ u equation
  {
    const double Z = -Zu[c];  // H_u = -(ax + ay + az) + nu lap
    // Z times the stencil factors, formed once, with the 1/2 of each two-point
    // average folded in (the sums below are twice the forward stencil's
    // averages): each contribution is then one multiply. The FP64 pipe bounds
    // this kernel; the atomics' additions happen in L2.
    const double Zx = Z * hx, Zy = Z * (0.5 * hy), Zz = Z * (0.5 * hz);
    const double u0 = u[c], uip = u[cip], uim = u[cim], ujp = u[cjp], ujm = u[cjm];
    const double ur = u0 + uip, ul = uim + u0;
    aadd(gu, cip, Zx * ur);
    aadd(gu, c, Zx * (ur - ul));
    aadd(gu, cim, -Zx * ul);
    const double Vj = v[cim] + v[c], Uj = ujm + u0;
    const double Vjp = v[ix(g, k, jp, im)] + v[cjp], Ujp = u0 + ujp;
    const double ZUjp = Zy * Ujp, ZUj = Zy * Uj;
    aadd(gv, ix(g, k, jp, im), ZUjp);
    aadd(gv, cjp, ZUjp);
    aadd(gv, cim, -ZUj);
    aadd(gv, c, -ZUj);
    aadd(gu, cjp, Zy * Vjp);
    aadd(gu, c, Zy * (Vjp - Vj));
    aadd(gu, cjm, -Zy * Vj);
    if (k > 0) {
      const double Wk = w[cim] + w[c], Uk = u[c - NXY] + u0;
      const double ZUk = Zz * Uk, ZWk = Zz * Wk;
      aadd(gw, cim, -ZUk);
      aadd(gw, c, -ZUk);
      aadd(gu, c - NXY, -ZWk);
      aadd(gu, c, -ZWk);
    }
    if (k < nz - 1) {
      const double Wk1 = w[cim + NXY] + w[c + NXY], Uk1 = u0 + u[c + NXY];
      const double ZUk1 = Zz * Uk1, ZWk1 = Zz * Wk1;
      aadd(gw, cim + NXY, ZUk1);
      aadd(gw, c + NXY, ZUk1);
      aadd(gu, c + NXY, ZWk1);
      aadd(gu, c, ZWk1);
    }
    const double Zl = Zu[c] * ph.nu;
    const double Zlx = Zl * g.rdx2, Zly = Zl * g.rdy2;
    aadd(gu, cip, Zlx);
    aadd(gu, cim, Zlx);
    aadd(gu, cjp, Zly);
    aadd(gu, cjm, Zly);
    aadd(gu, c, -2.0 * (Zlx + Zly));
    // direct terms: dt alpha (nu dzz u - G_x p)
    const double r = Ru[c] * da, rn = r * ph.nu, rx = r * rdx;
    aadd(gu, c, -rn * (m.cc[k] + m.ca[k]));
    if (k > 0) aadd(gu, c - NXY, rn * m.ca[k]);
    if (k < nz - 1) aadd(gu, c + NXY, rn * m.cc[k]);
    aadd(gp, c, -rx);
    aadd(gp, cim, rx);
  }
  // ------------------------------------------------------------ v equation
  {
    const double Z = -Zv[c];
    const double Zx = Z * (0.5 * hx), Zy = Z * hy, Zz = Z * (0.5 * hz);  // 1/2 folded in
    const double v0 = v[c], vip = v[cip], vim = v[cim], vjp = v[cjp], vjm = v[cjm];
    const double Uj = u[cjm] + u[c], Vj = vim + v0;
    const double Uip = u[ix(g, k, jm, ip)] + u[cip], Vip = v0 + vip;
    const double ZVip = Zx * Vip, ZVj = Zx * Vj;
    aadd(gu, ix(g, k, jm, ip), ZVip);
    aadd(gu, cip, ZVip);
    aadd(gu, cjm, -ZVj);
    aadd(gu, c, -ZVj);
    aadd(gv, cip, Zx * Uip);
    aadd(gv, c, Zx * (Uip - Uj));
    aadd(gv, cim, -Zx * Uj);
    const double vt = v0 + vjp, vb = vjm + v0;
    aadd(gv, cjp, Zy * vt);
    aadd(gv, c, Zy * (vt - vb));
    aadd(gv, cjm, -Zy * vb);
    if (k > 0) {
      const double Wk = w[cjm] + w[c], Vk = v[c - NXY] + v0;
      const double ZVk = Zz * Vk, ZWk = Zz * Wk;
      aadd(gw, cjm, -ZVk);
      aadd(gw, c, -ZVk);
      aadd(gv, c - NXY, -ZWk);
      aadd(gv, c, -ZWk);
    }
    if (k < nz - 1) {
      const double Wk1 = w[cjm + NXY] + w[c + NXY], Vk1 = v0 + v[c + NXY];
      const double ZVk1 = Zz * Vk1, ZWk1 = Zz * Wk1;
      aadd(gw, cjm + NXY, ZVk1);
      aadd(gw, c + NXY, ZVk1);
      aadd(gv, c + NXY, ZWk1);
      aadd(gv, c, ZWk1);
    }
    const double Zl = Zv[c] * ph.nu;
    const double Zlx = Zl * g.rdx2, Zly = Zl * g.rdy2;
    aadd(gv, cip, Zlx);
    aadd(gv, cim, Zlx);
    aadd(gv, cjp, Zly);
    aadd(gv, cjm, Zly);
    aadd(gv, c, -2.0 * (Zlx + Zly));
    const double r = Rv[c] * da, rn = r * ph.nu, ry = r * rdy;
    aadd(gv, c, -rn * (m.cc[k] + m.ca[k]));
    if (k > 0) aadd(gv, c - NXY, rn * m.ca[k]);
    if (k < nz - 1) aadd(gv, c + NXY, rn * m.cc[k]);
    aadd(gp, c, -ry);
    aadd(gp, cjm, ry);
  }
  if (k == 0) return;
  // ------------------------------------------------------------ w and T on face k
  const double wlo = m.wlo[k], whi = m.whi[k], rdzf = m.rdzf[k];
  const size_t ckm = c - NXY, cipkm = cip - NXY, cjpkm = cjp - NXY;
  const double ufi = wlo * u[ckm] + whi * u[c];
  const double ufip = wlo * u[cipkm] + whi * u[cip];
  const double vfj = wlo * v[ckm] + whi * v[c];
  const double vfjp = wlo * v[cjpkm] + whi * v[cjp];
  const double w0 = w[c], wk1 = w[c + NXY], wkm = w[ckm];
  const double wc_k = 0.5 * (w0 + wk1), wc_km = 0.5 * (wkm + w0);
  const bool up_int = k + 1 <= nz - 1, dn_int = k - 1 >= 1;  // neighbouring faces interior?
  {
    const double Z = -Zw[c];
    const double Zhx = Z * hx, Zhy = Z * hy, Zzf = Z * rdzf;
    const double wip = w[cip], wim = w[cim], wjp = w[cjp], wjm = w[cjm];
    // x: (ufip (w0+wip)/2 - ufi (wim+w0)/2)/dx
    const double a1 = Zhx * (w0 + wip), a0 = -Zhx * (wim + w0);
    aadd(gu, cipkm, a1 * wlo);
    aadd(gu, cip, a1 * whi);
    aadd(gu, ckm, a0 * wlo);
    aadd(gu, c, a0 * whi);
    aadd(gw, cip, Zhx * ufip);
    aadd(gw, c, Zhx * (ufip - ufi));
    aadd(gw, cim, -Zhx * ufi);
    const double b1 = Zhy * (w0 + wjp), b0 = -Zhy * (wjm + w0);
    aadd(gv, cjpkm, b1 * wlo);
    aadd(gv, cjp, b1 * whi);
    aadd(gv, ckm, b0 * wlo);
    aadd(gv, c, b0 * whi);
    aadd(gw, cjp, Zhy * vfjp);
    aadd(gw, c, Zhy * (vfjp - vfj));
    aadd(gw, cjm, -Zhy * vfj);
    // z: (wc_k^2 - wc_km^2)/dzf
    if (up_int) aadd(gw, c + NXY, Zzf * wc_k);
    aadd(gw, c, Zzf * (wc_k - wc_km));
    if (dn_int) aadd(gw, ckm, -Zzf * wc_km);
    const double Zl = Zw[c] * ph.nu;
    const double Zlx = Zl * g.rdx2, Zly = Zl * g.rdy2;
    aadd(gw, cip, Zlx);
    aadd(gw, cim, Zlx);
    aadd(gw, cjp, Zly);
    aadd(gw, cjm, Zly);
    aadd(gw, c, -2.0 * (Zlx + Zly));
    if (T) aadd(gT, c, Zw[c] * ph.buoy);
    const double r = Rw[c] * da, rn = r * ph.nu, rz = r * rdzf;
    aadd(gw, c, -rn * (m.fc[k] + m.fa[k]));
    if (dn_int) aadd(gw, ckm, rn * m.fa[k]);
    if (up_int) aadd(gw, c + NXY, rn * m.fc[k]);
    aadd(gp, c, -rz);
    aadd(gp, ckm, rz);
  }
  if (T) {
    const double Z = -ZT[c];
    const double Zhx = Z * hx, Zhy = Z * hy, Zhzf = Z * (0.5 * rdzf);
    const double t0 = T[c], tip = T[cip], tim = T[cim], tjp = T[cjp], tjm = T[cjm];
    const double tk1 = T[c + NXY], tkm = T[ckm];
    const double a1 = Zhx * (t0 + tip), a0 = -Zhx * (tim + t0);
    aadd(gu, cipkm, a1 * wlo);
    aadd(gu, cip, a1 * whi);
    aadd(gu, ckm, a0 * wlo);
    aadd(gu, c, a0 * whi);
    aadd(gT, cip, Zhx * ufip);
    aadd(gT, c, Zhx * (ufip - ufi));
    aadd(gT, cim, -Zhx * ufi);
    const double b1 = Zhy * (t0 + tjp), b0 = -Zhy * (tjm + t0);
    aadd(gv, cjpkm, b1 * wlo);
    aadd(gv, cjp, b1 * whi);
    aadd(gv, ckm, b0 * wlo);
    aadd(gv, c, b0 * whi);
    aadd(gT, cjp, Zhy * vfjp);
    aadd(gT, c, Zhy * (vfjp - vfj));
    aadd(gT, cjm, -Zhy * vfj);
    // z: (wc_k (t0+tk1)/2 - wc_km (tkm+t0)/2)/dzf
    const double tc_k = 0.5 * (t0 + tk1), tc_km = 0.5 * (tkm + t0);
    if (up_int) aadd(gw, c + NXY, Zhzf * tc_k);
    aadd(gw, c, Zhzf * (tc_k - tc_km));
    if (dn_int) aadd(gw, ckm, -Zhzf * tc_km);
    if (up_int) aadd(gT, c + NXY, Zhzf * wc_k);
    aadd(gT, c, Zhzf * (wc_k - wc_km));
    if (dn_int) aadd(gT, ckm, -Zhzf * wc_km);
    const double Zl = ZT[c] * ph.kappa;
    const double Zlx = Zl * g.rdx2, Zly = Zl * g.rdy2;
    aadd(gT, cip, Zlx);
    aadd(gT, cim, Zlx);
    aadd(gT, cjp, Zly);
    aadd(gT, cjm, Zly);
    aadd(gT, c, -2.0 * (Zlx + Zly));
    const double r = RT[c] * da, rk = r * ph.kappa;
    aadd(gT, c, -rk * (m.fc[k] + m.fa[k]));
    if (dn_int) aadd(gT, ckm, rk * m.fa[k]);
    if (up_int) aadd(gT, c + NXY, rk * m.fc[k]);
  }
}

__global__ void k_zero_walls(Grid g, double* a, double* b) {
  const size_t NXY = (size_t)g.nx * g.ny;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= NXY) return;
  if (a) {
    a[t] = 0.0;
    a[t + (size_t)g.nz * NXY] = 0.0;
  }
  if (b) {
    b[t] = 0.0;
    b[t + (size_t)g.nz * NXY] = 0.0;
  }
}

cudaError_t adjoint_explicit(afid_ctx* c, int l, double dt, const double* u, const double* v,
                             const double* w, const double* T, double* gu, double* gv, double* gw,
                             double* gT, double* gp, double* gHu, double* gHv, double* gHw,
                             double* gHT) {
  ProfScope ps(c, KF_ADJ);
  const Grid& g = c->g;
  int bx;
  dim3 grd = pgrid(g, bx);
  cudaError_t e;
  // wall planes of gw, gT are not unknowns
  k_zero_walls<<<ceil_div((long long)g.nx * g.ny, 256), 256, 0, c->stream>>>(g, gw, gT);
  k_adj_z<<<grd, bx, 0, c->stream>>>(g, gHu, gHv, gHw, T ? gHT : nullptr, c->R[0], c->R[1], c->R[2],
                                     c->R[3], dt * rk_gamma(l), 0);
  PhysA ph{c->phys.nu, c->phys.kappa, c->phys.buoyancy};
  k_adj_explicit<<<grd, bx, 0, c->stream>>>(g, c->m, ph, l, dt, u, v, w, T, gHu, gHv, gHw, gHT,
                                            c->R[0], c->R[1], c->R[2], c->R[3], gu, gv, gw, gT, gp);
  k_adj_z<<<grd, bx, 0, c->stream>>>(g, gHu, gHv, gHw, T ? gHT : nullptr, c->R[0], c->R[1], c->R[2],
                                     c->R[3], dt * rk_rho(l), 1);
  k_zero_walls<<<ceil_div((long long)g.nx * g.ny, 256), 256, 0, c->stream>>>(g, gw, gT);
  c->launches += 5;
  if ((e = cudaGetLastError())) return e;
  return cudaSuccess;
}

}  // namespace afid
