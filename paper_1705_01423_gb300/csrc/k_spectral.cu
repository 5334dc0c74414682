// Spectral stages of the Poisson solve (Sec. 2.2): forward real-to-complex FFT
// along x (optionally fused with the divergence of Sec. 2.2 step 1), complex
// FFT along y, one Thomas solve per (kx, ky) with modified wavenumbers,
// exact integration of the singular (0,0) mode, inverse FFTs.
//
// Spectral layout: spec[z][ky][kx], kx = 0..nx/2 in a row of pitch P complex
// elements. The x-transform reads contiguous rows, the y-transform stages a
// [ny] x [TK columns] tile in shared memory, and the Thomas sweep runs one
// system per thread with threads along kx, so every global access is coalesced
// and no global transpose is ever made (the paper's pencil transposes become
// this choice of layout).
#include "afid_internal.cuh"

namespace afid {

// --------------------------------------------------------------------------
// Thomas factor table, FP64: for every (kyh, kx) the reciprocal pivots
// m_k = 1 / (b_k - a_k c'_{k-1}), c'_k = c_k m_k, b_k = -a_k - c_k - lambda,
// lambda = lambda_x(kx) + lambda_y(kyh). Precomputed once, so the per-solve
// sweeps contain no division.
__global__ void k_thomas_table(Grid g, Metric m, const double* __restrict__ lamx,
                               const double* __restrict__ lamy, double* __restrict__ mtab64,
                               float* __restrict__ mtab32) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int kyh = blockIdx.y;
  const int W = g.M + 1;
  if (kx >= W) return;
  const size_t tplane = (size_t)g.nyh * W;
  double* out = mtab64 + (size_t)kyh * W + kx;
  float* out32 = mtab32 ? mtab32 + (size_t)kyh * W + kx : nullptr;
  if (kx == 0 && kyh == 0) {  // singular mode: handled by the exact prefix-sum kernel
    for (int k = 0; k < g.nz; ++k) {
      out[k * tplane] = 0.0;
      if (out32) out32[k * tplane] = 0.0f;
    }
    return;
  }
  const double lam = lamx[kx] + lamy[kyh];
  double cprev = 0.0;
  for (int k = 0; k < g.nz; ++k) {
    const double b = -m.pa[k] - m.pc[k] - lam;
    const double mk = 1.0 / (b - m.pa[k] * cprev);
    cprev = m.pc[k] * mk;
    out[k * tplane] = mk;
    if (out32) out32[k * tplane] = (float)mk;
  }
}

cudaError_t init_thomas_tables(afid_ctx* c) {
  const Grid& g = c->g;
  dim3 blk(128), grd(ceil_div(g.M + 1, 128), g.nyh);
  k_thomas_table<<<grd, blk, 0, c->stream>>>(g, c->m, c->lamx, c->lamy, c->mtab64, c->mtab32);
  c->launches++;
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Forward x transform. MODE_RHS: line = scale * src row; MODE_DIV: line =
// scale * D(u, v, w) on the fly. One block holds LINES rows; each row of nx
// reals is packed as nx/2 complex values z_n = x_2n + i x_2n+1, transformed
// with an nx/2-point FFT and unpacked into X_k, k = 0..nx/2:
//   E_k = (Z_k + conj Z_{M-k})/2, O_k = (Z_k - conj Z_{M-k})/(2i),
//   X_k = E_k + w_k O_k,  X_{M-k} = conj(E_k - w_k O_k),  w_k = exp(-2 pi i k/nx).
enum { MODE_RHS = 0, MODE_DIV = 1 };

template <typename R, int MODE>
__global__ void __launch_bounds__(512) k_r2c_x(Grid g, Metric m, const double* __restrict__ src,
                                               const double* __restrict__ u,
                                               const double* __restrict__ v,
                                               const double* __restrict__ w, double scale,
                                               typename cplx<R>::T* __restrict__ spec,
                                               const typename cplx<R>::T* __restrict__ tw,
                                               double* scal, int want_stats,
                                               const double* __restrict__ skip, int dev_s) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  if (dev_s) scale = 1.0 / scal[S_PROJ_S];
  const int M = g.M, T = M / 8;
  const int lines = blockDim.x / T;
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int nrows = g.nz * g.ny;
  const int row = blockIdx.x * lines + line;
  const bool active = row < nrows;
  const int stride = pad8(M) + 1;
  C* buf = sm + line * stride;
  double amax = 0.0;
  if (active) {
    const int nx = g.nx;
    if (MODE == MODE_RHS) {
      const double2* s2 = reinterpret_cast<const double2*>(src + (size_t)row * nx);
      for (int n = t; n < M; n += T) {
        double2 x = s2[n];
        x.x *= scale;
        x.y *= scale;
        if (want_stats) amax = fmax(amax, fmax(fabs(x.x), fabs(x.y)));
        buf[pad8(n)] = C{(R)x.x, (R)x.y};
      }
    } else {
      const int k = row / g.ny, j = row - (row / g.ny) * g.ny;
      const int jp = (j + 1) & (g.ny - 1);
      const double* ur = u + (size_t)row * nx;
      const double* vr = v + (size_t)row * nx;
      const double* vrp = v + ((size_t)k * g.ny + jp) * nx;
      const double* wr = w + (size_t)row * nx;
      const double* wrp = wr + (size_t)g.ny * nx;
      const double rdzc = m.rdzc[k];
      for (int n = t; n < M; n += T) {
        const int i = 2 * n;
        const double2 uu = *reinterpret_cast<const double2*>(ur + i);
        const double u2 = ur[(i + 2) & (nx - 1)];
        const double2 v0 = *reinterpret_cast<const double2*>(vr + i);
        const double2 v1 = *reinterpret_cast<const double2*>(vrp + i);
        const double2 w0 = *reinterpret_cast<const double2*>(wr + i);
        const double2 w1 = *reinterpret_cast<const double2*>(wrp + i);
        double d0 = (uu.y - uu.x) * g.rdx + (v1.x - v0.x) * g.rdy + (w1.x - w0.x) * rdzc;
        double d1 = (u2 - uu.y) * g.rdx + (v1.y - v0.y) * g.rdy + (w1.y - w0.y) * rdzc;
        d0 *= scale;
        d1 *= scale;
        if (want_stats) amax = fmax(amax, fmax(fabs(d0), fabs(d1)));
        buf[pad8(n)] = C{(R)d0, (R)d1};
      }
    }
  }
  __syncthreads();
  fft_line<false>(buf, M, tw, 2, t, active);
  if (active) {
    C* out = spec + (size_t)row * g.P;
    const R half = (R)0.5;
    for (int k = t; k <= M / 2; k += T) {
      const C zk = buf[pad8(k)];
      if (k == 0) {
        out[0] = C{zk.x + zk.y, (R)0};
        out[M] = C{zk.x - zk.y, (R)0};
        continue;
      }
      const C zm = buf[pad8(M - k)];
      const C E = C{(zk.x + zm.x) * half, (zk.y - zm.y) * half};
      const C O = C{(zk.y + zm.y) * half, (zm.x - zk.x) * half};
      const C wO = cmul(O, tw[k]);
      out[k] = cadd(E, wO);
      if (k != M / 2) out[M - k] = cconj(csub(E, wO));
    }
  }
  if (want_stats) {
    // block max of |rhs| -> one atomic per warp
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(scal + S_RHS_ABSMAX), dbl_key(amax));
  }
}

// --------------------------------------------------------------------------
// Inverse x transform: X_k, k = 0..M -> nx reals (imaginary parts of X_0 and
// X_M are ignored). Z'_k = E'_k + i O'_k with E'_k = X_k + conj X_{M-k},
// O'_k = (X_k - conj X_{M-k}) conj(w_k); an inverse M-point FFT gives
// nx (x_2n + i x_2n+1) before the 1/(nx ny) normalisation `scale`.
// ACC = 0 writes phi, ACC = 1 adds to phi.
template <typename R, int MODE>
__global__ void __launch_bounds__(512) k_c2r_x(Grid g, Metric m,
                                               const typename cplx<R>::T* __restrict__ spec,
                                               const typename cplx<R>::T* __restrict__ tw,
                                               double scale, double* __restrict__ phi,
                                               const double* __restrict__ skip,
                                               double* __restrict__ part) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int M = g.M, T = M / 8;
  const int lines = blockDim.x / T;
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int nrows = g.nz * g.ny;
  const int row = blockIdx.x * lines + line;
  const bool active = row < nrows;
  const int stride = pad8(M) + 1;
  C* buf = sm + line * stride;
  if (active) {
    const C* in = spec + (size_t)row * g.P;
    for (int k = t; k <= M; k += T) buf[pad8(k)] = in[k];
  }
  __syncthreads();
  if (active) {
    for (int k = t; k <= M / 2; k += T) {
      if (k == 0) {
        const R x0 = buf[pad8(0)].x, xm = buf[pad8(M)].x;
        buf[pad8(0)] = C{x0 + xm, x0 - xm};
        continue;
      }
      const C a = buf[pad8(k)], b = buf[pad8(M - k)];
      const C E = C{a.x + b.x, a.y - b.y};
      const C O = cmulc(C{a.x - b.x, a.y + b.y}, tw[k]);
      // Z'_k = E + i O ; Z'_{M-k} = conj(E) + i conj(O)
      buf[pad8(k)] = C{E.x - O.y, E.y + O.x};
      if (k != M / 2) buf[pad8(M - k)] = C{E.x + O.y, O.x - E.y};
    }
  }
  __syncthreads();
  fft_line<true>(buf, M, tw, 2, t, active);
  R d2 = (R)0;
  double psum = 0.0;
  if (active) {
    double2* o2 = reinterpret_cast<double2*>(phi + (size_t)row * g.nx);
    const R sc = (R)scale;
    for (int n = t; n < M; n += T) {
      const C z = buf[pad8(n)];
      if (MODE == 0) {
        o2[n] = make_double2((double)z.x * scale, (double)z.y * scale);
      } else {
        const R dx = z.x * sc, dy = z.y * sc;
        d2 += dx * dx + dy * dy;
        double2 r = make_double2((double)dx, (double)dy);
        if (MODE == 1) {
          const double2 old = o2[n];
          r.x += old.x;
          r.y += old.y;
        }
        psum += r.x + r.y;
        o2[n] = r;
      }
    }
    psum *= m.dzc[row / g.ny];
  }
  if (MODE != 0) {
    // per-block ||delta||^2 and sum of dzc * phi (weighted mean of phi)
    __shared__ double red[2][16];
    double dd = (double)d2;
    for (int o = 16; o > 0; o >>= 1) {
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
      psum += __shfl_xor_sync(0xffffffffu, psum, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = dd;
      red[1][threadIdx.x >> 5] = psum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
        a += red[0][wi];
        b += red[1][wi];
      }
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
  }
}

// --------------------------------------------------------------------------
// Complex FFT along y for a tile of TK consecutive kx columns of one z plane.
template <typename R, bool INV, int TK>
__global__ void __launch_bounds__(1024) k_fft_y(Grid g, typename cplx<R>::T* __restrict__ spec,
                                                const typename cplx<R>::T* __restrict__ tw,
                                                const double* __restrict__ skip) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int Ny = g.ny, T = Ny / 8;
  const int z = blockIdx.y, kx0 = blockIdx.x * TK;
  const int ncol = min(TK, g.M + 1 - kx0);
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int stride = pad8(Ny) + 1;
  C* base = spec + (size_t)z * Ny * g.P + kx0;
  for (int e = threadIdx.x; e < Ny * TK; e += blockDim.x) {
    const int ky = e / TK, c = e - (e / TK) * TK;
    if (c < ncol) sm[c * stride + pad8(ky)] = base[(size_t)ky * g.P + c];
  }
  __syncthreads();
  fft_line<INV>(sm + line * stride, Ny, tw, 1, t, line < ncol);
  for (int e = threadIdx.x; e < Ny * TK; e += blockDim.x) {
    const int ky = e / TK, c = e - (e / TK) * TK;
    if (c < ncol) base[(size_t)ky * g.P + c] = sm[c * stride + pad8(ky)];
  }
}

// --------------------------------------------------------------------------
// Thomas sweeps, one (kx, ky) system per thread (Sec. 2.2; the paper's GPU
// code also solves one system per thread, Sec. 3.2). Forward elimination
// d'_k = (d_k - a_k d'_{k-1}) m_k stored in place, back substitution
// x_k = d'_k - c_k m_k x_{k+1}. The (0,0) mode is left to k_zero_mode; in
// mixed precision the low modes (lambda < lam_thr) are left to k_thomas_low.
template <typename R>
__global__ void __launch_bounds__(128) k_thomas(Grid g, Metric m, typename cplx<R>::T* __restrict__ spec,
                                                const R* __restrict__ mtab,
                                                const R* __restrict__ pa, const R* __restrict__ pc,
                                                const double* __restrict__ lamx,
                                                const double* __restrict__ lamy, double lam_thr,
                                                const double* __restrict__ skip) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int ky = blockIdx.y;
  const int W = g.M + 1;
  if (kx >= W || (kx == 0 && ky == 0)) return;
  const int kyh = min(ky, g.ny - ky);
  if (lam_thr > 0.0 && lamx[kx] + lamy[kyh] < lam_thr) return;
  const size_t plane = (size_t)g.ny * g.P;
  const size_t tplane = (size_t)g.nyh * W;
  C* col = spec + (size_t)ky * g.P + kx;
  const R* mt = mtab + (size_t)kyh * W + kx;
  const int nz = g.nz;
  C d = col[0];
  R mk = mt[0];
  C dp = C{d.x * mk, d.y * mk};
  col[0] = dp;
#pragma unroll 4
  for (int k = 1; k < nz; ++k) {
    d = col[k * plane];
    mk = mt[k * tplane];
    const R ak = pa[k];
    dp = C{(d.x - ak * dp.x) * mk, (d.y - ak * dp.y) * mk};
    col[k * plane] = dp;
  }
  C x = dp;
#pragma unroll 4
  for (int k = nz - 2; k >= 0; --k) {
    const C e = col[k * plane];
    const R cp = pc[k] * mt[k * tplane];
    x = C{e.x - cp * x.x, e.y - cp * x.y};
    col[k * plane] = x;
  }
}

// Mixed precision: FP32 sweeps for most modes; the nearly singular low modes
// (lowslot[ky][kx] >= 0) are eliminated in FP64 with the FP64 pivot table,
// their intermediate d' kept in an FP64 scratch column [nz][nlow].
__global__ void __launch_bounds__(128) k_thomas_mixed(Grid g, Metric m, float2* __restrict__ spec,
                                                      const float* __restrict__ mtab32,
                                                      const double* __restrict__ mtab64,
                                                      const float* __restrict__ pa32,
                                                      const float* __restrict__ pc32,
                                                      const int* __restrict__ lowslot, int nlow,
                                                      double2* __restrict__ scratch,
                                                      const double* __restrict__ skip) {
  if (skip && *skip != 0.0) return;
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int ky = blockIdx.y;
  const int W = g.M + 1;
  if (kx >= W || (kx == 0 && ky == 0)) return;
  const int kyh = min(ky, g.ny - ky);
  const size_t plane = (size_t)g.ny * g.P;
  const size_t tplane = (size_t)g.nyh * W;
  float2* col = spec + (size_t)ky * g.P + kx;
  const int nz = g.nz;
  const int slot = lowslot[(size_t)ky * W + kx];
  if (slot < 0) {
    const float* mt = mtab32 + (size_t)kyh * W + kx;
    float2 d = col[0];
    float mk = mt[0];
    float2 dp = make_float2(d.x * mk, d.y * mk);
    col[0] = dp;
#pragma unroll 4
    for (int k = 1; k < nz; ++k) {
      d = col[k * plane];
      mk = mt[k * tplane];
      const float ak = pa32[k];
      dp = make_float2((d.x - ak * dp.x) * mk, (d.y - ak * dp.y) * mk);
      col[k * plane] = dp;
    }
    float2 x = dp;
#pragma unroll 4
    for (int k = nz - 2; k >= 0; --k) {
      const float2 e = col[k * plane];
      const float cp = pc32[k] * mt[k * tplane];
      x = make_float2(e.x - cp * x.x, e.y - cp * x.y);
      col[k * plane] = x;
    }
    return;
  }
  const double* mt = mtab64 + (size_t)kyh * W + kx;
  double2 dp = make_double2(0.0, 0.0);
  for (int k = 0; k < nz; ++k) {
    const float2 d = col[k * plane];
    const double mk = mt[k * tplane];
    const double ak = m.pa[k];
    dp = make_double2(((double)d.x - ak * dp.x) * mk, ((double)d.y - ak * dp.y) * mk);
    scratch[(size_t)k * nlow + slot] = dp;
  }
  double2 x = dp;
  col[(size_t)(nz - 1) * plane] = make_float2((float)x.x, (float)x.y);
  for (int k = nz - 2; k >= 0; --k) {
    const double2 e = scratch[(size_t)k * nlow + slot];
    const double cp = m.pc[k] * mt[k * tplane];
    x = make_double2(e.x - cp * x.x, e.y - cp * x.y);
    col[k * plane] = make_float2((float)x.x, (float)x.y);
  }
}

// --------------------------------------------------------------------------
// Exact solution of the singular (0,0) mode in FP64 (one block): remove the
// dzc-weighted mean of bhat (solvability), flux prefix sums
// F_{k+1} = F_k + dzc_k bhat_k, phi_k = phi_{k-1} + dzf_k F_k, then the gauge
// (zero dzc-weighted mean). Also records the removed mean of the rhs.
template <typename R>
__global__ void k_zero_mode(Grid g, Metric m, typename cplx<R>::T* __restrict__ spec, double* scal,
                            const double* __restrict__ skip) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ double zb[];
  const int nz = g.nz;
  const size_t plane = (size_t)g.ny * g.P;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) zb[k] = (double)spec[k * plane].x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sw = 0.0, sb = 0.0;
    for (int k = 0; k < nz; ++k) {
      sw += m.dzc[k];
      sb += m.dzc[k] * zb[k];
    }
    const double mu = sb / sw;
    scal[S_RHS_MEAN] = mu / ((double)g.nx * (double)g.ny);
    double F = 0.0, ph = 0.0, sp = 0.0;
    double bprev = zb[0] - mu;
    zb[0] = 0.0;
    for (int k = 1; k < nz; ++k) {
      F += m.dzc[k - 1] * bprev;
      bprev = zb[k] - mu;
      ph += m.dzf[k] * F;
      zb[k] = ph;
      sp += m.dzc[k] * ph;
    }
    const double pm = sp / sw;
    for (int k = 0; k < nz; ++k) zb[k] -= pm;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nz; k += blockDim.x) spec[k * plane] = C{(R)zb[k], (R)0};
}

// --------------------------------------------------------------------------
template <typename R>
static int r2c_lines(const Grid& g) {
  const int T = g.M / 8;
  int lines = 256 / T;
  if (lines < 1) lines = 1;
  return lines;
}

template <typename R>
static size_t line_smem(int N) {
  return (size_t)(pad8(N) + 1) * sizeof(typename cplx<R>::T);
}

template <typename R>
static cudaError_t run_fft_y(afid_ctx* c, typename cplx<R>::T* spec, const typename cplx<R>::T* tw,
                             bool inv, const double* skip) {
  ProfScope ps(c, KF_FFTY);
  const Grid& g = c->g;
  const size_t ls = line_smem<R>(g.ny);
  // widest tile that keeps a block within 1024 threads and ~112 KB of shared memory
  int tk = 8;
  while (tk > 1 && ((size_t)tk * ls > 112 * 1024 || tk * (g.ny / 8) > 1024)) tk /= 2;
  dim3 grd(ceil_div(g.M + 1, tk), g.nz);
  const int thr = tk * (g.ny / 8);
  const size_t sm = (size_t)tk * ls;
#define AFID_FFTY(TKV)                                                                        \
  do {                                                                                        \
    auto kf = inv ? k_fft_y<R, true, TKV> : k_fft_y<R, false, TKV>;                          \
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);           \
    kf<<<grd, thr, sm, c->stream>>>(g, spec, tw, skip);                                      \
  } while (0)
  switch (tk) {
    case 8: AFID_FFTY(8); break;
    case 4: AFID_FFTY(4); break;
    case 2: AFID_FFTY(2); break;
    default: AFID_FFTY(1); break;
  }
#undef AFID_FFTY
  c->launches++;
  return cudaGetLastError();
}

template <typename R>
static cudaError_t run_r2c(afid_ctx* c, const double* rhs, const double* u, const double* v,
                           const double* w, bool dev_s, typename cplx<R>::T* spec,
                           const typename cplx<R>::T* tw, int want_stats, const double* skip) {
  const double scale = 1.0;
  ProfScope ps(c, KF_R2C);
  const Grid& g = c->g;
  const int T = g.M / 8, lines = r2c_lines<R>(g);
  const size_t sm = (size_t)lines * line_smem<R>(g.M);
  const int blocks = ceil_div((long long)g.nz * g.ny, lines);
  if (rhs) {
    auto kf = k_r2c_x<R, MODE_RHS>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, rhs, u, v, w, scale, spec, tw, c->scal,
                                             want_stats, skip, (int)dev_s);
  } else {
    auto kf = k_r2c_x<R, MODE_DIV>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, rhs, u, v, w, scale, spec, tw, c->scal,
                                             want_stats, skip, (int)dev_s);
  }
  c->launches++;
  return cudaGetLastError();
}

template <typename R>
static cudaError_t run_c2r(afid_ctx* c, const typename cplx<R>::T* spec,
                           const typename cplx<R>::T* tw, double* phi, int mode,
                           const double* skip, double* part) {
  ProfScope ps(c, KF_C2R);
  const Grid& g = c->g;
  const int T = g.M / 8, lines = r2c_lines<R>(g);
  const size_t sm = (size_t)lines * line_smem<R>(g.M);
  const int blocks = ceil_div((long long)g.nz * g.ny, lines);
  const double scale = 1.0 / ((double)g.nx * (double)g.ny);
  auto kf = mode == 1 ? k_c2r_x<R, 1> : (mode == 2 ? k_c2r_x<R, 2> : k_c2r_x<R, 0>);
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, spec, tw, scale, phi, skip, part);
  c->launches++;
  return cudaGetLastError();
}

// Direct FP64 solve: phi = L^-1 (src / s) with src = rhs (rhs != NULL) or the
// divergence of (u, v, w); s = S_PROJ_S when dev_s, else 1.
cudaError_t spectral_solve(afid_ctx* c, const double* rhs, const double* u, const double* v,
                           const double* w, bool dev_s, double* phi, bool want_stats) {
  const Grid& g = c->g;
  double2* spec = static_cast<double2*>(c->spec);
  cudaError_t e;
  if ((e = run_r2c<double>(c, rhs, u, v, w, dev_s, spec, c->twx64, want_stats, nullptr))) return e;
  if ((e = run_fft_y<double>(c, spec, c->twy64, false, nullptr))) return e;
  {
    ProfScope ps(c, KF_THOMAS);
    dim3 grd(ceil_div(g.M + 1, 128), g.ny);
    k_thomas<double><<<grd, 128, 0, c->stream>>>(g, c->m, spec, c->mtab64, c->m.pa, c->m.pc,
                                                 c->lamx, c->lamy, 0.0, nullptr);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
  }
  {
    ProfScope ps(c, KF_ZERO);
    k_zero_mode<double><<<1, 256, g.nz * sizeof(double), c->stream>>>(g, c->m, spec, c->scal, nullptr);
  }
  c->launches++;
  if ((e = cudaGetLastError())) return e;
  if ((e = run_fft_y<double>(c, spec, c->twy64, true, nullptr))) return e;
  return run_c2r<double>(c, spec, c->twx64, phi, 0, nullptr, nullptr);
}

// FP32 spectral solve of `src` (FP64) for the mixed-precision refinement:
// phi = delta (first) or phi += delta, with per-block partials of ||delta||^2
// and of sum dzc phi in c->part2; every kernel returns at once when *skip != 0.
cudaError_t spectral_solve_fp32(afid_ctx* c, const double* src, double* phi, const double* skip,
                                bool first) {
  const Grid& g = c->g;
  float2* spec = static_cast<float2*>(c->spec);
  cudaError_t e;
  if ((e = run_r2c<float>(c, src, nullptr, nullptr, nullptr, false, spec, c->twx32, 0, skip))) return e;
  if ((e = run_fft_y<float>(c, spec, c->twy32, false, skip))) return e;
  {
    ProfScope ps(c, KF_THOMAS);
    dim3 grd(ceil_div(g.M + 1, 128), g.ny);
    k_thomas_mixed<<<grd, 128, 0, c->stream>>>(g, c->m, spec, c->mtab32, c->mtab64, c->pa32,
                                               c->pc32, c->lowslot, c->nlow, c->low_scratch, skip);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
  }
  {
    ProfScope ps(c, KF_ZERO);
    k_zero_mode<float><<<1, 256, g.nz * sizeof(double), c->stream>>>(g, c->m, spec, c->scal, skip);
  }
  c->launches++;
  if ((e = cudaGetLastError())) return e;
  if ((e = run_fft_y<float>(c, spec, c->twy32, true, skip))) return e;
  return run_c2r<float>(c, spec, c->twx32, phi, first ? 2 : 1, skip, c->part2);
}

}  // namespace afid

namespace afid {
int c2r_blocks(const Grid& g) {
  const int T = g.M / 8;
  int lines = 256 / T;
  if (lines < 1) lines = 1;
  return ceil_div((long long)g.nz * g.ny, lines);
}
}  // namespace afid
