// Physical-space stages: projection and pressure update (Sec. 2.2 last
// paragraph), divergence check, CFL (Listing 1), the explicit terms of the
// RK3 substep with the right-hand side of its Crank-Nicolson systems (Sec.
// 2.1), the wall-normal Crank-Nicolson sweeps, and the FP64 residual and
// norms of the mixed-precision refinement.
//
// Stencil kernels run one thread per grid point with x along threadIdx.x, so
// every neighbour load of a warp is a contiguous 256-byte row segment (the
// x +- 1 neighbours hit L1). The wall-normal sweeps run one thread per (x, y)
// column and walk z, again coalesced across x.
#include "afid_internal.cuh"

namespace afid {

__device__ __forceinline__ size_t at(const Grid& g, int k, int j, int i) {
  return ((size_t)k * g.ny + j) * g.nx + i;
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// integer maximum (ordered bit patterns of non-negative doubles)
template <> __device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum, result valid in thread 0 (blockDim.x multiple of 32, <= 1024)
__device__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

static inline dim3 point_grid(const Grid& g, int nzp, int& bx) {
  bx = x_block(g.nx, 128);
  return dim3(g.nx / bx, g.ny, nzp);
}

// ---------------------------------------------------------------------------
// Projection and pressure update:
//   u -= s (phi_i - phi_{i-1})/dx, v -= s (phi_j - phi_{j-1})/dy,
//   w_k -= s (phi_k - phi_{k-1})/dzf_k (interior faces),
//   p += phi - beta [pc_k (phi_{k+1} - phi_k) - pa_k (phi_k - phi_{k-1})]
//      = p + (1 + beta (pa_k + pc_k)) phi_k - beta pc_k phi_{k+1} - beta pa_k phi_{k-1}
// (pa_0 = pc_{nz-1} = 0: zero-flux walls). One thread per (x, y) column
// marches over a chunk of k with phi_{k-1}, phi_k, phi_{k+1} in registers;
// the per-row factors are formed once per block in shared memory, which
// leaves 9 FP64 operations per point (this part issues 2 FP64 operations per
// clock per SM, so the count, not HBM, sets the time).
__global__ void __launch_bounds__(256) k_project(Grid g, Metric m, double* __restrict__ u,
                                                 double* __restrict__ v, double* __restrict__ w,
                                                 double* __restrict__ p, const double* __restrict__ phi,
                                                 const double* __restrict__ scal, int kchunk) {
  extern __shared__ double pco[];  // [4][kchunk]: s/dzf, 1 + beta (pa + pc), beta pc, beta pa
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * blockDim.x + tx, j = blockIdx.y * blockDim.y + ty;
  const int k0 = blockIdx.z * kchunk, k1 = min(g.nz, k0 + kchunk);
  const double s = scal[S_PROJ_S], beta = scal[S_PROJ_BETA];
  double* sz = pco;
  double* bd = pco + kchunk;
  double* bc = pco + 2 * kchunk;
  double* ba = pco + 3 * kchunk;
  for (int q = ty * blockDim.x + tx; q < k1 - k0; q += blockDim.x * blockDim.y) {
    const int k = k0 + q;
    sz[q] = s * m.rdzf[k];
    const double bpc = beta * m.pc[k], bpa = beta * m.pa[k];
    bc[q] = bpc;
    ba[q] = bpa;
    bd[q] = 1.0 + (bpc + bpa);
  }
  __syncthreads();
  const double sx = s * g.rdx, sy = s * g.rdy;
  const size_t NXY = (size_t)g.nx * g.ny;
  const int im = wrap_prev(i, g.nx), jm = wrap_prev(j, g.ny);
  const size_t col = (size_t)j * g.nx + i, cim = (size_t)j * g.nx + im, cjm = (size_t)jm * g.nx + i;
  size_t c = (size_t)k0 * NXY;
  double f = phi[c + col];
  double fkm = k0 > 0 ? phi[c - NXY + col] : f;
#pragma unroll 2
  for (int k = k0; k < k1; ++k, c += NXY) {
    const int q = k - k0;
    const double fkp = k < g.nz - 1 ? phi[c + NXY + col] : f;
    const double fim = phi[c + cim], fjm = phi[c + cjm];
    u[c + col] = fma(-sx, f - fim, u[c + col]);
    v[c + col] = fma(-sy, f - fjm, v[c + col]);
    if (k > 0) w[c + col] = fma(-sz[q], f - fkm, w[c + col]);
    if (p) {
      double pv = fma(bd[q], f, p[c + col]);
      pv = fma(-bc[q], fkp, pv);
      pv = fma(-ba[q], fkm, pv);
      p[c + col] = pv;
    }
    fkm = f;
    f = fkp;
  }
}

cudaError_t project(afid_ctx* c, double* u, double* v, double* w, double* p, const double* phi) {
  ProfScope ps(c, KF_PROJECT);
  const Grid& g = c->g;
  const int bx = x_block(g.nx, 32), by = 8;
  // chunks of k so that the grid is several waves of resident blocks
  const long long bxy = (long long)(g.nx / bx) * (g.ny / by);
  const long long want = 32LL * c->num_sms;
  int nch = (int)((want + bxy - 1) / bxy);
  const int max_ch = g.nz / 8 > 0 ? g.nz / 8 : 1;
  nch = nch < 1 ? 1 : (nch > max_ch ? max_ch : nch);
  const int min_ch = (g.nz + 1023) / 1024;  // shared memory <= 32 KB per block
  nch = nch < min_ch ? min_ch : nch;
  const int kchunk = (g.nz + nch - 1) / nch;
  nch = (g.nz + kchunk - 1) / kchunk;
  dim3 blk(bx, by), grd(g.nx / bx, g.ny / by, nch);
  k_project<<<grd, blk, (size_t)4 * kchunk * sizeof(double), c->stream>>>(g, c->m, u, v, w, p, phi,
                                                                         c->scal, kchunk);
  c->launches++;
  return cudaGetLastError();
}

__global__ void k_set_proj(double* scal, double s, double beta) {
  scal[S_PROJ_S] = s;
  scal[S_PROJ_RS] = 1.0 / s;
  scal[S_PROJ_BETA] = beta;
}

cudaError_t set_proj_scalars(afid_ctx* c, double s, double beta) {
  ProfScope ps(c, KF_PROJECT);
  k_set_proj<<<1, 1, 0, c->stream>>>(c->scal, s, beta);
  c->launches++;
  return cudaGetLastError();
}

// b = D(u, v, w) / s (the divergence of Sec. 2.2 step 1), s = S_PROJ_S
__global__ void k_div(Grid g, Metric m, const double* __restrict__ u, const double* __restrict__ v,
                      const double* __restrict__ w, double* __restrict__ b,
                      const double* __restrict__ scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const double rs = scal[S_PROJ_RS];
  const size_t c = at(g, k, j, i);
  const int ip = wrap_next(i, g.nx), jp = wrap_next(j, g.ny);
  const double d = (u[at(g, k, j, ip)] - u[c]) * g.rdx + (v[at(g, k, jp, i)] - v[c]) * g.rdy +
                   (w[c + (size_t)g.nx * g.ny] - w[c]) * m.rdzc[k];
  b[c] = d * rs;
}

cudaError_t divergence_to(afid_ctx* c, const double* u, const double* v, const double* w, double* b) {
  ProfScope ps(c, KF_PROJECT);
  int bx;
  dim3 grd = point_grid(c->g, c->g.nz, bx);
  k_div<<<grd, bx, 0, c->stream>>>(c->g, c->m, u, v, w, b, c->scal);
  c->launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// max |D u| over cells (grid-stride, one atomic per warp)
__global__ void k_maxdiv(Grid g, Metric m, const double* __restrict__ u,
                         const double* __restrict__ v, const double* __restrict__ w,
                         unsigned long long* out) {
  double mx = 0.0;
  // rows (k, j) across blocks, x across threads: no 64-bit division per point
  for (int row = blockIdx.x; row < g.nz * g.ny; row += gridDim.x) {
    const int k = row / g.ny, j = row - k * g.ny;
    const int jp = wrap_next(j, g.ny);
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const size_t c = (size_t)row * g.nx + i;
      const int ip = wrap_next(i, g.nx);
      const double d = (u[at(g, k, j, ip)] - u[c]) * g.rdx + (v[at(g, k, jp, i)] - v[c]) * g.rdy +
                       (w[c + (size_t)g.nx * g.ny] - w[c]) * m.rdzc[k];
      mx = fmax(mx, fabs(d));
    }
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, dbl_key(mx));
}

cudaError_t max_divergence(afid_ctx* c, const double* u, const double* v, const double* w,
                           double* out_dev) {
  ProfScope ps(c, KF_CFL);
  cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double), c->stream);
  if (e) return e;
  k_maxdiv<<<c->num_sms * 8, 256, 0, c->stream>>>(c->g, c->m, u, v, w,
                                                  reinterpret_cast<unsigned long long*>(out_dev));
  c->launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CFL of Listing 1: 0.5 max(|u_i+u_i+1|/dx + |v_j+v_j+1|/dy + |w_k+w_k+1|/dzc_k),
// floored at 1e-8; dt = min(cfl/cflm, dt_max). The terms are non-negative, so
// their maximum is taken on the bit patterns with integer instructions (off the
// FP64 pipe that bounds the kernel: 6 FP64 operations per point, not 7); a NaN
// velocity gives a NaN CFL number.
__global__ void k_cfl(Grid g, Metric m, const double* __restrict__ u, const double* __restrict__ v,
                      const double* __restrict__ w, unsigned long long* out) {
  unsigned long long mx = 0ull;
  for (int row = blockIdx.x; row < g.nz * g.ny; row += gridDim.x) {
    const int k = row / g.ny, j = row - k * g.ny;
    const int jp = wrap_next(j, g.ny);
    const double rz = m.rdzc[k];
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const size_t c = (size_t)row * g.nx + i;
      const int ip = wrap_next(i, g.nx);
      const double q = fabs(u[c] + u[at(g, k, j, ip)]) * g.rdx + fabs(v[c] + v[at(g, k, jp, i)]) * g.rdy +
                       fabs(w[c] + w[c + (size_t)g.nx * g.ny]) * rz;
      mx = max(mx, dbl_key(q));
    }
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx > 0ull) atomicMax(out, mx);
}

__global__ void k_cfl_final(double* scal, double cfl, double dt_max, double* cflm_dev) {
  const double q = __longlong_as_double((long long)reinterpret_cast<unsigned long long*>(scal)[S_CFLM]);
  const double cflm = fmax(1e-8, 0.5 * q);
  if (cflm_dev) *cflm_dev = cflm;
  scal[S_CFLM] = cflm;
  scal[S_DT] = fmin(cfl / cflm, dt_max);
}

cudaError_t cfl(afid_ctx* c, const double* u, const double* v, const double* w, double cflv,
                double dt_max, double* cflm_dev) {
  ProfScope ps(c, KF_CFL);
  cudaError_t e = cudaMemsetAsync(c->scal + S_CFLM, 0, sizeof(double), c->stream);
  if (e) return e;
  k_cfl<<<c->num_sms * 8, 256, 0, c->stream>>>(c->g, c->m, u, v, w,
                                               reinterpret_cast<unsigned long long*>(c->scal + S_CFLM));
  k_cfl_final<<<1, 1, 0, c->stream>>>(c->scal, cflv, dt_max, cflm_dev);
  c->launches += 2;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Crank-Nicolson factor tables for substep l: operator o = 0 (cells, nu),
// 1 (faces, nu), 2 (faces, kappa); (I - beta dzz) with beta = alpha_l dt d/2.
// Row k: sub = -beta a_k, diag = 1 + beta (a_k + c_k), sup = -beta c_k;
// tab[o][0][k] = sub_k, tab[o][1][k] = m_k = 1/(diag_k - sub_k c'_{k-1}),
// tab[o][2][k] = c'_k = sup_k m_k, tab[o][3][k] = sup_k; for the explicit
// side of the same substep (the alpha_l dt d dzz q term of R) tab[o][4][k] =
// 2 beta a_k, tab[o][5][k] = 2 beta c_k, tab[o][6][k] = -2 beta (a_k + c_k).
// Thread 0 also publishes dt, the projection scale s = alpha_l dt and
// beta = alpha_l dt nu/2.
// One warp per variable set o. The coefficients of every row are independent
// and computed by all lanes. The pivots follow from the continuant
// Q_k = diag_k Q_{k-1} - sub_k sup_{k-1} Q_{k-2} (Q_{k0-1} = 1, Q_{k0-2} = 0):
// m_k = 1 / (diag_k - sub_k c'_{k-1}) = Q_{k-1} / Q_k and c'_k = sup_k m_k.
// Its serial chain is one FMA per row (the product with Q_{k-2} is formed a
// row ahead), run by one lane with a power-of-two rescaling every 8 rows;
// the divisions then run in parallel over the rows. (On this part a
// dependent FP64 operation costs tens of cycles, and a division in the chain
// of the direct recurrence several of them per row.)
__global__ void __launch_bounds__(96) k_cn_tables(Grid g, Metric m, int l, double dt_in,
                                                  double* __restrict__ scal, double nu, double kappa,
                                                  double* __restrict__ tab) {
  const int o = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double dt = dt_in > 0.0 ? dt_in : scal[S_DT];
  if (threadIdx.x == 0) {
    scal[S_DT] = dt;
    scal[S_PROJ_S] = rk_alpha(l) * dt;
    scal[S_PROJ_RS] = 1.0 / (rk_alpha(l) * dt);
    scal[S_PROJ_BETA] = rk_alpha(l) * dt * nu * 0.5;
  }
  if (o >= 3) return;
  const double beta = rk_alpha(l) * dt * (o == 2 ? kappa : nu) * 0.5;
  const int L = g.nz + 1;
  double* sub = tab + (size_t)o * CN_TAB_ARRAYS * L;
  double* mm = sub + L;
  double* cp = mm + L;
  double* sp = cp + L;
  double* ea = sp + L;   // explicit-side alpha_l dt d dzz coefficients (RHS)
  double* ec = ea + L;
  double* ed = ec + L;
  const int k0 = o == 0 ? 0 : 1, k1 = g.nz;  // rows k0..nz-1
  const double* __restrict__ pa = o == 0 ? m.ca : m.fa;
  const double* __restrict__ pc = o == 0 ? m.cc : m.fc;
  if (o == 0) {  // per-plane factors of the explicit terms (k_rhs_zm)
    double* pz = ed + L;
    const double adt = rk_alpha(l) * dt;
    for (int k = lane; k < L; k += 32) {
      pz[k] = adt * m.rdzf[k];
      pz[L + k] = k < g.nz ? 0.25 * m.rdzc[k] : 0.0;
      pz[2 * L + k] = 0.25 * m.rdzf[k];
    }
  }
  // every row's coefficients; diag_k -> mm[k] and sub_k sup_{k-1} -> cp[k]
  // as the chain's inputs (both overwritten by it)
  for (int k = k0 + lane; k < k1; k += 32) {
    const double a = pa[k], c = pc[k];
    const double sk = -beta * a;
    sub[k] = sk;
    sp[k] = -beta * c;
    const double xa = 2.0 * beta * a, xc = 2.0 * beta * c;
    ea[k] = xa;
    ec[k] = xc;
    ed[k] = -(xa + xc);
    mm[k] = 1.0 + beta * (a + c);
    cp[k] = k > k0 ? sk * (-beta * pc[k - 1]) : 0.0;
  }
  __syncwarp();
  if (lane == 0) {
    // continuant chain; Q_{k-1} -> mm[k], Q_k -> cp[k] (same scale). A warp
    // FP64 instruction costs the same with one active lane, so the chain
    // holds only its own two operations per row; its inputs are loaded a
    // batch of B rows ahead.
    constexpr int B = 16;
    double dA[B], gA[B], dB[B], gB[B];
    auto load_batch = [&](int kb, double* dd, double* gg) {
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int k = kb + q < k1 ? kb + q : k1 - 1;
        dd[q] = mm[k];
        gg[q] = cp[k];
      }
    };
    load_batch(k0, dA, gA);
    double q1 = 1.0, q2 = 0.0;
    for (int kb = k0; kb < k1; kb += B) {
      if (kb + B < k1) load_batch(kb + B, dB, gB);
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int k = kb + q;
        if (k < k1) {
          if (((k - k0) & 7) == 0) {  // rescale q1, q2 by 2^-e, |q1| = f 2^e, f in [0.5, 1)
            const long long bits = __double_as_longlong(q1);
            const int e = (int)((bits >> 52) & 0x7ff) - 1022;
            const double sc = __longlong_as_double((long long)(1023 - e) << 52);
            q1 *= sc;
            q2 *= sc;
          }
          const double qn = fma(dA[q], q1, -(gA[q] * q2));
          mm[k] = q1;
          cp[k] = qn;
          q2 = q1;
          q1 = qn;
        }
      }
#pragma unroll
      for (int q = 0; q < B; ++q) {
        dA[q] = dB[q];
        gA[q] = gB[q];
      }
    }
  }
  __syncwarp();
  const double adt = rk_alpha(l) * dt, gdt = rk_gamma(l) * dt, rdt = rk_rho(l) * dt;
  double* const base = tab + (size_t)o * CN_TAB_ARRAYS * L;
  for (int k = k0 + lane; k < k1; k += 32) {
    const double mk = mm[k] / cp[k];
    mm[k] = mk;
    cp[k] = sp[k] * mk;
    // the coefficients of the right-hand side scaled by the reciprocal pivot
    base[CN_MSUB * L + k] = mk * sub[k];
    base[CN_MEA * L + k] = mk * ea[k];
    base[CN_MEC * L + k] = mk * ec[k];
    base[CN_MED * L + k] = mk * ed[k];
    base[CN_MCG * L + k] = mk * gdt;
    base[CN_MCR * L + k] = mk * rdt;
    if (o == 0) {
      base[CN_MGX * L + k] = mk * (adt * g.rdx);
      base[CN_MGY * L + k] = mk * (adt * g.rdy);
    } else if (o == 1) {
      base[CN_MGX * L + k] = mk * (adt * m.rdzf[k]);
    }
  }
}

cudaError_t cn_tables(afid_ctx* c, int l, double dt) {
  ProfScope ps(c, KF_CNTAB);
  k_cn_tables<<<1, 96, 0, c->stream>>>(c->g, c->m, l, dt, c->scal, c->phys.nu, c->phys.kappa,
                                       c->cntab);
  c->launches++;
  return cudaGetLastError();
}

// One thread per (x, y) column of variable blockIdx.y (0 u, 1 v, 2 w, 3 T);
// cells k = 0..nz-1 for u, v, interior faces k = 1..nz-1 for w, T.
// Forward (ADJ = false): elimination writes d' over R, back substitution adds
// dq = A^-1 R to q. Transposed (ADJ = true): R = A^-T q with A = L U from the
// same factors (U: diagonal 1/m_k, superdiagonal sup_k; L: unit, subdiagonal
// sub_k m_{k-1}), solving U^T z = q forward and L^T y = z backward; q is kept.
template <bool ADJ>
__global__ void k_cn_sweep(Grid g, const double* __restrict__ tab, double* R0, double* R1,
                           double* R2, double* R3, double* q0, double* q1, double* q2, double* q3) {
  const int var = blockIdx.y;
  double* R = var == 0 ? R0 : var == 1 ? R1 : var == 2 ? R2 : R3;
  double* q = var == 0 ? q0 : var == 1 ? q1 : var == 2 ? q2 : q3;
  if (!q) return;
  const size_t NXY = (size_t)g.nx * g.ny;
  const size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (col >= NXY) return;
  const int o = var < 2 ? 0 : (var == 2 ? 1 : 2);
  const int L = g.nz + 1;
  const double* sub = tab + (size_t)o * CN_TAB_ARRAYS * L;
  const double* mm = sub + L;
  const double* cp = mm + L;
  const double* sp = cp + L;
  const int k0 = var < 2 ? 0 : 1, k1 = g.nz - 1;  // inclusive range
  if (!ADJ) {
    // R holds m_k R_k (the explicit-terms kernels scale it): d'_k0 = R_k0 and
    // d'_k = R_k - (m_k sub_k) d'_{k-1}, one FMA per row
    const double* msub = sub + (size_t)CN_MSUB * L;
    double dp = R[k0 * NXY + col];
    for (int k = k0 + 1; k <= k1; ++k) {
      dp = fma(-msub[k], dp, R[k * NXY + col]);
      R[k * NXY + col] = dp;
    }
    // q += x is issued as an atomic addition (each location is updated once, by
    // this thread, so the result is that of the plain addition): the addition
    // is done in L2, off the FP64 pipe that bounds this sweep, and q is not
    // loaded by the SM
    double x = dp;
    atomicAdd(q + k1 * NXY + col, x);
    for (int k = k1 - 1; k >= k0; --k) {
      x = R[k * NXY + col] - cp[k] * x;
      atomicAdd(q + k * NXY + col, x);
    }
  } else {
    double z = q[k0 * NXY + col] * mm[k0];
    R[k0 * NXY + col] = z;
    for (int k = k0 + 1; k <= k1; ++k) {
      z = (q[k * NXY + col] - sp[k - 1] * z) * mm[k];
      R[k * NXY + col] = z;
    }
    double y = z;
    for (int k = k1 - 1; k >= k0; --k) {
      y = R[k * NXY + col] - sub[k + 1] * mm[k] * y;
      R[k * NXY + col] = y;
    }
  }
}

cudaError_t cn_sweeps(afid_ctx* c, double* u, double* v, double* w, double* T) {
  ProfScope ps(c, KF_CN);
  const size_t NXY = (size_t)c->g.nx * c->g.ny;
  dim3 grd(ceil_div((long long)NXY, 128), 4);
  k_cn_sweep<false><<<grd, 128, 0, c->stream>>>(c->g, c->cntab, c->R[0], c->R[1], c->R[2], c->R[3],
                                                u, v, w, T);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t cn_tables_grid(const Grid& g, const Metric& m, int l, double dt, double* scal, double nu,
                           double kappa, double* tab, cudaStream_t st) {
  k_cn_tables<<<1, 96, 0, st>>>(g, m, l, dt, scal, nu, kappa, tab);
  return cudaGetLastError();
}

cudaError_t cn_sweep_scalar(const Grid& g, const double* tab, double* RT, double* T, cudaStream_t st) {
  const size_t NXY = (size_t)g.nx * g.ny;
  dim3 grd(ceil_div((long long)NXY, 128), 4);  // the blocks of variables 0-2 return at once
  k_cn_sweep<false><<<grd, 128, 0, st>>>(g, tab, nullptr, nullptr, nullptr, RT, nullptr, nullptr,
                                         nullptr, T);
  return cudaGetLastError();
}

cudaError_t cn_sweeps_adjoint(afid_ctx* c, double* gu, double* gv, double* gw, double* gT) {
  ProfScope ps(c, KF_CN);
  const size_t NXY = (size_t)c->g.nx * c->g.ny;
  dim3 grd(ceil_div((long long)NXY, 128), 4);
  k_cn_sweep<true><<<grd, 128, 0, c->stream>>>(c->g, c->cntab, c->R[0], c->R[1], c->R[2], c->R[3],
                                               gu, gv, gw, gT);
  c->launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Mixed-precision refinement. FP64 statistics of b, FP64 residual
// r = (b - mean_W b) - L phi, the convergence test on the correction norms,
// and the final FP64 gauge (zero weighted mean of phi: the residual cannot
// see a constant, so the FP32 corrections' gauge round-off is removed here).
// ---------------------------------------------------------------------------
// Wall-normal statistics (Sec. 3.2: statistics accumulated only along the
// wall-normal direction, a vector reduction; Sec. 5: Nusselt number, wall
// shear stress and friction Reynolds number). One block per face plane
// k = 0..nz forms the horizontal means
//   0 <u>  1 <v>  2 <u^2>  3 <v^2>            (cell plane k < nz)
//   4 <w>  5 <w^2>  6 <T>  7 <T^2>  8 <w T>   (face plane k)
// with per-thread partial sums in a fixed order (compensated for the first
// moments) and the block sum added by warp 0 (deterministic).
// prof: [nz+1][AFID_STAT_NQ].
__global__ void __launch_bounds__(256) k_plane_stats(Grid g, const double* __restrict__ u,
                                                     const double* __restrict__ v,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ T,
                                                     double* __restrict__ prof) {
  constexpr int NQ = AFID_STAT_NQ;
  __shared__ double red[NQ][256];
  const int k = blockIdx.x;
  const size_t NXY = (size_t)g.nx * g.ny;
  const size_t c0 = (size_t)k * NXY;
  double s[NQ];
  double e0 = 0.0, e1 = 0.0, e4 = 0.0, e6 = 0.0;  // compensations of the first moments
#pragma unroll
  for (int q = 0; q < NQ; ++q) s[q] = 0.0;
  const bool cell = k < g.nz;
  for (size_t c = threadIdx.x; c < NXY; c += blockDim.x) {
    if (cell) {
      const double a = u[c0 + c], b = v[c0 + c];
      two_sum_acc(s[0], e0, a);
      two_sum_acc(s[1], e1, b);
      s[2] = fma(a, a, s[2]);
      s[3] = fma(b, b, s[3]);
    }
    const double ww = w[c0 + c];
    two_sum_acc(s[4], e4, ww);
    s[5] = fma(ww, ww, s[5]);
    if (T) {
      const double t = T[c0 + c];
      two_sum_acc(s[6], e6, t);
      s[7] = fma(t, t, s[7]);
      s[8] = fma(ww, t, s[8]);
    }
  }
  // the means enter differences across a wall cell (wall Nusselt numbers,
  // wall shear stress), so their sums are compensated
  s[0] += e0;
  s[1] += e1;
  s[4] += e4;
  s[6] += e6;
#pragma unroll
  for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int q = 0; q < NQ; ++q) {
      double t = 0.0;
      for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) t += red[q][i];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) prof[(size_t)k * NQ + q] = t / (double)NXY;
    }
  }
}

// Scalars from the profiles (one thread; formulas of afid_stats in afid.h):
// out[0..6] = nu_volume, nu_bottom, nu_top, tau_bottom, tau_top, re_tau, ke.
__global__ void k_stats_scalars(Grid g, Metric m, afid_phys ph, const double* __restrict__ prof,
                                double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  constexpr int NQ = AFID_STAT_NQ;
  const int nz = g.nz;
  double height = 0.0, wT = 0.0, kuv = 0.0, kw = 0.0;
  for (int k = 0; k < nz; ++k) {
    height += m.dzc[k];
    kuv += m.dzc[k] * (prof[k * NQ + 2] + prof[k * NQ + 3]);
  }
  for (int k = 1; k < nz; ++k) {
    wT += m.dzf[k] * prof[k * NQ + 8];
    kw += m.dzf[k] * prof[k * NQ + 5];
  }
  const double dT = ph.T_bot - ph.T_top;
  out[0] = ph.kappa > 0.0 ? 1.0 + (wT / height) / ph.kappa : 0.0;
  out[1] = dT != 0.0 ? -(prof[1 * NQ + 6] - prof[0 * NQ + 6]) / m.dzc[0] / dT : 0.0;
  out[2] = dT != 0.0 ? -(prof[nz * NQ + 6] - prof[(nz - 1) * NQ + 6]) / m.dzc[nz - 1] / dT : 0.0;
  out[3] = ph.nu * (prof[0] - ph.u_bot) / (0.5 * m.dzc[0]);
  out[4] = ph.nu * (ph.u_top - prof[(nz - 1) * NQ]) / (0.5 * m.dzc[nz - 1]);
  const double u_tau = sqrt(0.5 * (fabs(out[3]) + fabs(out[4])));
  out[5] = ph.nu > 0.0 ? 0.5 * height * u_tau / ph.nu : 0.0;
  out[6] = 0.5 * (kuv + kw) / height;
}

cudaError_t statistics_grid(const Grid& g, const Metric& m, const afid_phys& ph, const double* u,
                            const double* v, const double* w, const double* T, double* stat_buf,
                            cudaStream_t st) {
  k_plane_stats<<<g.nz + 1, 256, 0, st>>>(g, u, v, w, T, stat_buf);
  k_stats_scalars<<<1, 32, 0, st>>>(g, m, ph, stat_buf, stat_buf + (size_t)(g.nz + 1) * AFID_STAT_NQ);
  return cudaGetLastError();
}

cudaError_t statistics(afid_ctx* c, const double* u, const double* v, const double* w, const double* T) {
  c->launches += 2;
  return statistics_grid(c->g, c->m, c->phys, u, v, w, T, c->stat_buf, c->stream);
}

// Volume Nusselt number (Sec. 5, Table 3; volume form Nu = 1 + coef <w T>_V
// with coef = sqrt(Ra Pr) in free-fall units) and, when gw / gT are given, its
// derivatives dNu/dw = f_k T and dNu/dT = f_k w with f_k = coef dx dy dzf_k / V
// on the interior faces (zero on the walls) -- the cotangent seeds of the
// adjoint rollout. One block per face plane k = 0..nz; the plane sum of w T
// (interior planes) is formed in a fixed order and added by warp 0 into
// psum[k] (deterministic), then k_nusselt_final adds dzf_k psum[k] over k.
__global__ void __launch_bounds__(256) k_nusselt_planes(Grid g, Metric m, const double* __restrict__ w,
                                                         const double* __restrict__ T, double fscale,
                                                         double* __restrict__ gw, double* __restrict__ gT,
                                                         double* __restrict__ psum) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  const size_t NXY = (size_t)g.nx * g.ny;
  const size_t c0 = (size_t)k * NXY;
  const bool interior = k > 0 && k < g.nz;
  const double f = interior ? fscale * m.dzf[k] : 0.0;
  double s = 0.0;
  for (size_t c = threadIdx.x; c < NXY; c += blockDim.x) {
    const double ww = w[c0 + c], t = T[c0 + c];
    if (interior) s = fma(ww, t, s);
    if (gw) gw[c0 + c] = f * t;
    if (gT) gT[c0 + c] = f * ww;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) t += red[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) psum[k] = t;
  }
}

// Nu = 1 + (coef dx dy / V) sum_k dzf_k psum[k] over the interior planes, one
// lane, fixed order.
__global__ void k_nusselt_final(Grid g, Metric m, const double* __restrict__ psum, double fscale,
                                double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 1; k < g.nz; ++k) s = fma(m.dzf[k], psum[k], s);
  out[0] = 1.0 + fscale * s;
}

cudaError_t nusselt(afid_ctx* c, const double* w, const double* T, double coef, double* gw,
                    double* gT) {
  ProfScope ps(c, KF_ADJ);
  const Grid& g = c->g;
  double height = 0.0;
  for (int k = 0; k < g.nz; ++k) height += c->zf_host[k + 1] - c->zf_host[k];
  const double fscale = coef * g.dx * g.dy / (c->lx * c->ly * height);
  double* psum = c->stat_buf;  // nz + 1 plane sums, then Nu
  k_nusselt_planes<<<g.nz + 1, 256, 0, c->stream>>>(g, c->m, w, T, fscale, gw, gT, psum);
  k_nusselt_final<<<1, 32, 0, c->stream>>>(g, c->m, psum, fscale, psum + (g.nz + 1));
  c->launches += 2;
  return cudaGetLastError();
}

// Reduction of the per-block partials of the first mixed-precision forward
// transform (k_r2c_x32<R32_FIRST>): weighted mean of b and ||b - mean||^2;
// resets the refinement's scalars.
// hz: sum of dzc (formed on the host: a serial loop of nz dependent FP64 adds
// in one thread would cost the kernel more than its reduction).
__global__ void k_bstats_final(Grid g, double hz, const double* part, int np, double* scal) {
  double sw = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    sw += part[3 * i];
    s1 += part[3 * i + 1];
    s2 += part[3 * i + 2];
  }
  sw = block_sum(sw);
  s1 = block_sum(s1);
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    const double n = (double)g.nx * (double)g.ny * (double)g.nz;
    const double mean = sw / (hz * (double)g.nx * (double)g.ny);
    scal[S_BMEAN] = mean;
    scal[S_BNORM2] = s2 - 2.0 * mean * s1 + n * mean * mean;
    scal[S_RNORM2] = scal[S_BNORM2];
    scal[S_ITERS] = 0.0;
    scal[S_DNORM2] = 0.0;
    scal[S_ERREST] = 1.0;
    scal[S_PHIMEAN] = 0.0;
  }
}

cudaError_t bstats_final(afid_ctx* c) {
  ProfScope ps(c, KF_REFINE);
  k_bstats_final<<<1, 1024, 0, c->stream>>>(c->g, c->hz, c->part3, c2r_blocks(c->g), c->scal);
  c->launches++;
  return cudaGetLastError();
}

// Convergence test after correction k (iterations counted here). The stopping
// rule uses the correction norms: with linear convergence the error left after
// correction k >= 3 is about ||d_k|| (||d_k|| / ||d_{k-1}||), after correction
// 2 at most ||d_2||; ||d_1|| stands for ||phi||. (A residual test alone
// under-estimates the error by up to the condition number of L.) Also records
// the weighted mean of phi and the norm of the residual computed before this
// correction.
__global__ void k_refine_check(Grid g, double hz, const double* part, int np, const double* part2,
                               int np2, double* scal, double tol) {
  if (scal[S_CONVERGED] != 0.0) return;
  double d2 = 0.0, ps = 0.0, rs = 0.0;
  for (int i = threadIdx.x; i < np2; i += blockDim.x) {
    d2 += part2[2 * i];
    ps += part2[2 * i + 1];
  }
  const bool have_r = scal[S_ITERS] > 0.5;
  if (have_r)
    for (int i = threadIdx.x; i < np; i += blockDim.x) rs += part[3 * i];
  d2 = block_sum(d2);
  ps = block_sum(ps);
  rs = block_sum(rs);
  if (threadIdx.x == 0) {
    // every accumulate pass removes the mean measured after the previous one
    // and sums dzc * delta_k: the weighted mean of phi is now that of delta_k
    const double dm = ps / (hz * (double)g.nx * (double)g.ny);
    scal[S_PHIMEAN] = dm;
    if (have_r) scal[S_RNORM2] = rs;
    scal[S_ITERS] += 1.0;
    const double k = scal[S_ITERS];
    const double prev = scal[S_DNORM2];
    if (k < 1.5) scal[S_D1NORM2] = d2;
    const double ref = scal[S_D1NORM2];
    // squared estimate. After correction 2 the bound is ||d_2|| itself: the
    // ratio ||d_2||/||d_1|| measures one FP32 solve of b, whose error sits in
    // the well-resolved large modes, and does not predict the solve of the
    // residual, whose error sits in the ill-conditioned low modes just above
    // the FP64 threshold (a ratio-based stop after correction 2 left 1.4e-10
    // on the 1024 x 512 x 256 plane Couette grid while predicting 7.6e-12).
    double est2;
    if (k < 2.5) est2 = d2;
    else est2 = prev > 0.0 ? d2 * d2 / prev : 0.0;
    scal[S_DPREV2] = prev;
    scal[S_DNORM2] = d2;
    scal[S_ERREST] = ref > 0.0 ? sqrt(est2 / ref) : 0.0;
    if (d2 == 0.0 || (k > 1.5 && est2 <= tol * tol * ref)) scal[S_CONVERGED] = 1.0;
  }
}

// Final FP64 gauge when the refinement stopped without converging (after a
// converged refinement the mean left is that of the last, tiny, correction's
// rounding and the kernel returns at once).
__global__ void k_sub_mean(Grid g, double* __restrict__ phi, const double* __restrict__ scal) {
  if (scal[S_CONVERGED] != 0.0) return;
  const size_t n2 = (size_t)g.nx * g.ny * g.nz / 2;  // nx is even
  const double pm = scal[S_PHIMEAN];
  double2* p2 = reinterpret_cast<double2*>(phi);
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n2;
       c += (size_t)gridDim.x * blockDim.x) {
    double2 v = p2[c];
    v.x -= pm;
    v.y -= pm;
    p2[c] = v;
  }
}

// Mixed-precision refined solve (device-side convergence test, no host sync):
//   k = 1: phi = FP32-solve(b), with the FP64 stats of b (mean_W b, ||b||)
//          taken in the same forward transform;
//   k = 2: phi += FP32-solve(r), r = (b - mean) - L phi in FP64, formed
//          inside the forward transform;
//   k = 3..max: phi += FP32-solve(r), r = r_prev - L delta_prev updated in
//          two-float arithmetic from the stored residual and correction;
//   after every correction: convergence test on the correction norms; the
//   gauge (zero weighted mean) is carried by the accumulate passes.
// Every kernel returns at once once the test has passed.
cudaError_t mixed_solve(afid_ctx* c, const double* b, double* phi, bool stats) {
  const Grid& g = c->g;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->scal + S_CONVERGED, 0, sizeof(double), c->stream))) return e;
  const int np2 = c->part2_len;
  for (int it = 0; it < c->max_iter; ++it) {
    if ((e = spectral_solve_fp32(c, b, phi, phi, c->scal + S_CONVERGED, it, stats))) return e;
    ProfScope ps(c, KF_REFINE);
    k_refine_check<<<1, 1024, 0, c->stream>>>(g, c->hz, c->part3, np2, c->part2, np2, c->scal, c->tol);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
  }
  ProfScope ps(c, KF_REFINE);
  k_sub_mean<<<c->part_len, 256, 0, c->stream>>>(g, phi, c->scal);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace afid
