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
#include <algorithm>
#include <cmath>
#include <cstring>

#include "afid_internal.cuh"

namespace afid {

// --------------------------------------------------------------------------
// Thomas factor table, FP64: for every (kyh, kx) the reciprocal pivots
// m_k = 1 / (b_k - a_k c'_{k-1}), c'_k = c_k m_k, b_k = -a_k - c_k - lambda,
// lambda = lambda_x(kx) + lambda_y(kyh). Precomputed once, so the per-solve
// sweeps contain no division.
__global__ void k_thomas_table(Grid g, Metric m, const double* __restrict__ lamx,
                               const double* __restrict__ lamy, double* __restrict__ mtab64,
                               float* __restrict__ mtab32, float* __restrict__ mtabt32) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int kyh = blockIdx.y;
  const int W = g.M + 1;
  if (kx >= W) return;
  const size_t tplane = (size_t)g.nyh * W;
  double* out = mtab64 + (size_t)kyh * W + kx;
  float* out32 = mtab32 ? mtab32 + (size_t)kyh * W + kx : nullptr;
  // mtabt32 (fused small-nz solve): the FP32 table transposed to [kx][k][kyh]
  float* outt = mtabt32 ? mtabt32 + (size_t)kx * g.nz * g.nyh + kyh : nullptr;
  if (kx == 0 && kyh == 0) {  // singular mode: handled by the exact prefix-sum kernel
    for (int k = 0; k < g.nz; ++k) {
      out[k * tplane] = 0.0;
      if (out32) out32[k * tplane] = 0.0f;
      if (outt) outt[(size_t)k * g.nyh] = 0.0f;
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
    if (outt) outt[(size_t)k * g.nyh] = (float)mk;
  }
}

cudaError_t init_thomas_tables(afid_ctx* c) {
  const Grid& g = c->g;
  dim3 blk(128), grd(ceil_div(g.M + 1, 128), g.nyh);
  k_thomas_table<<<grd, blk, 0, c->stream>>>(g, c->m, c->lamx, c->lamy, c->mtab64, c->mtab32, c->mtabt32);
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

// FP64 -> working precision. For FP32 the value is truncated with integer
// operations (sign, rebiased exponent, top 23 mantissa bits; magnitudes below
// the FP32 normal range flush to zero, above it saturate) instead of a
// conversion instruction, which issues on the FP64 pipe; the refinement that
// consumes the FP32 solve corrects the truncation like any other FP32 error.
// FP32 -> FP64 widening with integer operations (exact for normal numbers and
// zero; FP32 subnormals flush to zero).
template <typename R> __device__ __forceinline__ double to_double(R x) { return (double)x; }
template <> __device__ __forceinline__ double to_double<float>(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long bits = sign | ((unsigned long long)(e + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// s += x with the exact rounding error of the addition (Knuth's TwoSum, with
// the round-to-nearest intrinsics so that no step is contracted or
// re-associated) added to the compensation c.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float xp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, xp)), __fsub_rn(x, xp));
  s = t;
  c = __fadd_rn(c, e);
}

// The part of x below its FP32 truncation to_real<float>(x), as an FP32
// number (integer operations and one integer-to-float conversion: the 29
// mantissa bits dropped by the truncation, scaled by 2^(e - 52), the scale a
// subnormal FP32 power of two for small |x|). to_real<float>(x) + low_part(x)
// equals x to about 2^-48 relative for |x| >= 2^-74, with gradually less
// precision in the tail below that.
__device__ __forceinline__ float low_part(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned lo29 = (unsigned)b & 0x1fffffffu;
  const int e = (int)((b >> 52) & 0x7ff);       // biased FP64 exponent
  const int fe = e - 1075 + 127;                // FP32 biased exponent of 2^(e - 1075)
  if (fe <= -23 || fe >= 255 || lo29 == 0u) return 0.f;
  const unsigned sb = fe > 0 ? (unsigned)fe << 23 : 1u << (fe + 22);
  const float mag = __uint2float_rn(lo29) * __uint_as_float(sb);
  return (b >> 63) ? -mag : mag;
}

// Two-float accumulation (sh, sl) += (ch + cl) v for an FP32 v: the product
// ch v is split exactly into p + pe (FMA), p is added by TwoSum, and the
// rounding errors with cl v and pe are collected in sl. Intrinsics keep every
// step as written.
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float ch, float cl, float v) {
  const float p = __fmul_rn(ch, v);
  const float pe = __fmaf_rn(ch, v, -p);
  const float t = __fadd_rn(sh, p);
  const float tp = __fsub_rn(t, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, tp)), __fsub_rn(p, tp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(e, __fmaf_rn(cl, v, pe)));
}

// (hi, lo) = a - b for two-float a, b, renormalised (|lo| <= ulp(hi)/2).
__device__ __forceinline__ float2 ff_sub(float ah, float al, float bh, float bl) {
  const float t = __fsub_rn(ah, bh);
  const float tp = __fsub_rn(t, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(t, tp)), __fsub_rn(-bh, tp));
  const float lo = __fadd_rn(e, __fsub_rn(al, bl));
  const float hi = __fadd_rn(t, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t)));
}

// Product rounded on its own (never fused into a following add).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename R> __device__ __forceinline__ R to_real(double x);
template <> __device__ __forceinline__ double to_real<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_real<float>(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ff) - 1023 + 127;
  const unsigned sign = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f7fffffu);
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

// TAN (FP64, power-of-two M >= 64): the M-point FFT's radix-8 passes take their
// twiddles in tangent form from `ttab` (tan_tables, forward, tlen doubles),
// copied over the per-pass table region.
template <typename R, int MODE, bool GEN, bool TAN = false>
__global__ void __launch_bounds__(512, TAN ? 2 : 0) k_r2c_x(Grid g, Metric m, const double* __restrict__ src,
                                               const double* __restrict__ u,
                                               const double* __restrict__ v,
                                               const double* __restrict__ w, double scale,
                                               typename cplx<R>::T* __restrict__ spec,
                                               const typename cplx<R>::T* __restrict__ tw,
                                               double* scal, int want_stats,
                                               const double* __restrict__ skip, int dev_s,
                                               const double* __restrict__ ttab, int tlen) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  if (dev_s) scale = scal[S_PROJ_RS];
  const int M = g.M, T = M / 8;
  const int lines = blockDim.x / T;
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int nrows = g.nz * g.ny;
  const int row = blockIdx.x * lines + line;
  const bool active = row < nrows;
  const int stride = pad8(M) + 1;
  C* buf = sm + line * stride;
  C* stw = sm + lines * stride;  // twiddle table, nx entries
  C* stp = stw + g.nx;           // per-pass tables of the M-point FFT (power-of-two M)
  C* stq = stp + (TAN ? max(M, (tlen + 1) / 2) : M);  // unpacking twiddles w_k / 2, k <= M/2
  for (int q = threadIdx.x; q < g.nx; q += blockDim.x) stw[q] = tw[q];
  if constexpr (TAN) {
    double* sd = reinterpret_cast<double*>(stp);
    for (int q = threadIdx.x; q < tlen; q += blockDim.x) sd[q] = ttab[q];
  } else if (!GEN) {
    pass_twiddles(stp, tw, M, 2, threadIdx.x, blockDim.x);
  }
  for (int q = threadIdx.x; q <= M / 2; q += blockDim.x) stq[q] = cscale(tw[q], (R)0.5);
  double amax = 0.0;
  if (active) {
    const int nx = g.nx;
    if (MODE == MODE_RHS) {
      const double2* s2 = reinterpret_cast<const double2*>(src + (size_t)row * nx);
      for (int n = t; n < M; n += T) {
        double2 x = s2[n];
        if (scale != 1.0) {
          x.x *= scale;
          x.y *= scale;
        }
        if (want_stats) amax = fmax(amax, fmax(fabs(x.x), fabs(x.y)));
        buf[pad8(n)] = C{to_real<R>(x.x), to_real<R>(x.y)};
      }
    } else {
      const int k = row / g.ny, j = row - (row / g.ny) * g.ny;
      const int jp = wrap_next(j, g.ny);
      const double* ur = u + (size_t)row * nx;
      const double* vr = v + (size_t)row * nx;
      const double* vrp = v + ((size_t)k * g.ny + jp) * nx;
      const double* wr = w + (size_t)row * nx;
      const double* wrp = wr + (size_t)g.ny * nx;
      // the scale (1/s) folded into the three inverse spacings
      const double sx = g.rdx * scale, sy = g.rdy * scale, sz = m.rdzc[k] * scale;
      for (int n = t; n < M; n += T) {
        const int i = 2 * n;
        const double2 uu = *reinterpret_cast<const double2*>(ur + i);
        const double u2 = ur[wrap_add(i, 2, nx)];
        const double2 v0 = *reinterpret_cast<const double2*>(vr + i);
        const double2 v1 = *reinterpret_cast<const double2*>(vrp + i);
        const double2 w0 = *reinterpret_cast<const double2*>(wr + i);
        const double2 w1 = *reinterpret_cast<const double2*>(wrp + i);
        const double d0 = fma(uu.y - uu.x, sx, fma(v1.x - v0.x, sy, (w1.x - w0.x) * sz));
        const double d1 = fma(u2 - uu.y, sx, fma(v1.y - v0.y, sy, (w1.y - w0.y) * sz));
        if (want_stats) amax = fmax(amax, fmax(fabs(d0), fabs(d1)));
        buf[pad8(n)] = C{(R)d0, (R)d1};
      }
    }
  }
  __syncthreads();
  if constexpr (GEN) fft_line<false, true>(buf, M, stw, 2, t, active);
  else if constexpr (TAN)  // launched for FP64 lines only (the cast is the identity there)
    fft_line_tan_ix<false>(reinterpret_cast<double2*>(buf), M, reinterpret_cast<const double*>(stp), t, active, PadIx{});
  else fft_line_pt<false>(buf, M, stp, t, active);
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
      // X_k = E + w_k O, X_M-k = conj(E - w_k O) with E = (Z_k + conj Z_M-k)/2,
      // O = (Z_k - conj Z_M-k)/(2i): the halves folded into the FMAs and
      // into the table (w_k / 2)
      const C E2 = C{zk.x + zm.x, zk.y - zm.y};
      const C wO = cmul(C{zk.y + zm.y, zm.x - zk.x}, stq[k]);
      out[k] = C{fma(half, E2.x, wO.x), fma(half, E2.y, wO.y)};
      if (k != M / 2) out[M - k] = C{fma(half, E2.x, -wO.x), fma(-half, E2.y, wO.y)};
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
// Mixed precision forward x transform: FP64 input line -> FP32 spectrum, no
// FP64 arithmetic per point except where the refinement needs it.
//   R32_FIRST: line = b. Per-block partial sums of dzc*b and b (and of b^2
//              and max |b| with stats) for the weighted mean removed from b
//              (solvability) and the reported norm: part[3 blk + 0..2]. The
//              row sums are compensated FP32 sums of the FP64 values split
//              into head and tail (about 2^-46 relative), b^2 in FP32.
//   R32_RESID: line = r = (b - mean_W b) - L phi, the refinement's FP64
//              residual, computed on the fly (7-point operator of Sec. 2.2;
//              8 FP64 operations per point); with stats the per-block ||r||^2
//              (FP32, report only) in part[3 blk].
//   R32_RESUPD: line = r_k = r_{k-1} - L delta_{k-1} (k >= 2), with
//              r_{k-1} the stored two-float residual and delta_{k-1} the FP32
//              correction the previous step added to phi; the 7-point sum in
//              two-float arithmetic (no FP64 operations). The error of this
//              update is a few 2^-46 of the stencil's terms, i.e. of
//              |r_{k-1}| times the local condition, far below the FP32
//              accuracy of the solve it feeds; r_k is stored back.
//   R32_RESUPD_ST: the same update with the block's stencil footprint staged
//              in shared memory first (cp.async, every load of the block in
//              flight at once): the block's rows are lines consecutive j of one
//              plane (ny a multiple of lines), so it needs the rows j0-1 ..
//              j0+lines of its plane and j0 .. j0+lines-1 of the planes below and
//              above, 3 lines + 2 rows of delta; same arithmetic, same results.
//              Blocks of at most 256 threads, three per SM.
// R32_RESID and R32_RESUPD store the residual as (head, tail) in rres.
// Same line transform and unpacking as k_r2c_x.
enum { R32_FIRST = 0, R32_RESID = 1, R32_RESUPD = 2, R32_RESUPD_ST = 3 };

// float2 words of dynamic shared memory in front of the twiddle table: the
// lines' transform buffers, which R32_RESUPD_ST lays over its staged rows.
__host__ __device__ __forceinline__ int r2c32_front_words(int mode, int lines, int nx, int stride) {
  const int b = lines * stride;
  if (mode != R32_RESUPD_ST) return b;
  const int st = ((3 * lines + 2) * nx + 1) / 2;
  return st > b ? st : b;
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// r - L delta at two neighbouring points (i, i+1) of a row in two-float
// arithmetic: f = (delta_i, delta_i+1), fw = delta_i-1, fe = delta_i+2, fn / fs
// the rows j+1 / j-1, fu / fd the planes k+1 / k-1 (used when up / dn), ro the
// stored residual (head_i, tail_i, head_i+1, tail_i+1); returns the new one.
__device__ __forceinline__ float4 resupd_pair(float2 f, float fw, float fe, float2 fn, float2 fs, float2 fu,
                                              float2 fd, bool up, bool dn, float4 ro, float2 ca, float2 cc,
                                              float2 cd, float xh, float xl, float yh, float yl) {
  // S = L delta = rdx2 (w + e) + rdy2 (s + n) + pc up + pa down - pdiag centre
  float sxh = 0.f, sxl = 0.f, syh = 0.f, syl = 0.f;
  ff_acc(sxh, sxl, -cd.x, -cd.y, f.x);
  ff_acc(syh, syl, -cd.x, -cd.y, f.y);
  ff_acc(sxh, sxl, xh, xl, fw);
  ff_acc(sxh, sxl, xh, xl, f.y);
  ff_acc(syh, syl, xh, xl, f.x);
  ff_acc(syh, syl, xh, xl, fe);
  ff_acc(sxh, sxl, yh, yl, fn.x);
  ff_acc(sxh, sxl, yh, yl, fs.x);
  ff_acc(syh, syl, yh, yl, fn.y);
  ff_acc(syh, syl, yh, yl, fs.y);
  if (up) {
    ff_acc(sxh, sxl, cc.x, cc.y, fu.x);
    ff_acc(syh, syl, cc.x, cc.y, fu.y);
  }
  if (dn) {
    ff_acc(sxh, sxl, ca.x, ca.y, fd.x);
    ff_acc(syh, syl, ca.x, ca.y, fd.y);
  }
  const float2 nx2 = ff_sub(ro.x, ro.y, sxh, sxl);
  const float2 ny2 = ff_sub(ro.z, ro.w, syh, syl);
  return make_float4(nx2.x, nx2.y, ny2.x, ny2.y);
}

// Block sum of one double per thread, valid on thread 0. The values go
// through shared memory (red: blockDim.x doubles) and only warp 0 adds them:
// on this part a warp FP64 instruction costs the same whatever its active
// lanes, so a shuffle tree in every warp would cost each warp five adds.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) t += red[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

template <int MODE, bool GEN>
__global__ void __launch_bounds__(MODE == R32_RESUPD_ST ? 256 : 512, MODE == R32_RESUPD_ST ? 3 : 0) k_r2c_x32(Grid g, Metric m, const double* __restrict__ b,
                                                 const double* __restrict__ phi, float2* __restrict__ spec,
                                                 const float2* __restrict__ tw, double* __restrict__ scal,
                                                 double* __restrict__ part, int stats,
                                                 const double* __restrict__ skip, float2* __restrict__ rres,
                                                 const float* __restrict__ dprev,
                                                 const float2* __restrict__ cff) {
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[512];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int M = g.M, T = M / 8;
  const int lines = blockDim.x / T;
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int nrows = g.nz * g.ny;
  const int row = blockIdx.x * lines + line;
  const bool active = row < nrows;
  const int stride = pad8(M) + 1;
  float2* buf = sm + line * stride;
  float2* stw = sm + r2c32_front_words(MODE, lines, g.nx, stride);  // twiddle table, nx entries
  float2* stp = stw + g.nx;  // per-pass tables of the M-point FFT (power-of-two M)
  for (int q = threadIdx.x; q < g.nx; q += blockDim.x) stw[q] = tw[q];
  if (!GEN) pass_twiddles(stp, tw, M, 2, threadIdx.x, blockDim.x);
  float fs = 0.f, fc = 0.f, fs2 = 0.f;  // FIRST: compensated FP32 row sum, sum of squares
  float2 zr[8];                         // FIRST: the thread's points, for the first FFT pass
  float rr = 0.f;
  unsigned long long amax = 0ull;
  int k = 0;
  if (MODE == R32_RESUPD_ST) {  // every row of the block is active
    const int nx = g.nx, q4 = nx >> 2;
    const int row0 = blockIdx.x * lines;
    k = row0 / g.ny;
    const int j0 = row0 - k * g.ny;
    // staged rows: 0 .. lines+1 plane k at j0-1 .. j0+lines (periodic in y),
    // lines+2 .. 2 lines+1 plane k-1, 2 lines+2 .. 3 lines+1 plane k+1
    float* st = reinterpret_cast<float*>(smem_raw);
    const int nst = (3 * lines + 2) * q4;
    for (int c = threadIdx.x; c < nst; c += blockDim.x) {
      const int r = c / q4, q = c - r * q4;
      int kk = k, jj;
      if (r < lines + 2) {
        jj = j0 - 1 + r;
        jj = jj < 0 ? jj + g.ny : (jj >= g.ny ? jj - g.ny : jj);
      } else if (r < 2 * lines + 2) {
        kk = k - 1;
        jj = j0 + r - (lines + 2);
      } else {
        kk = k + 1;
        jj = j0 + r - (2 * lines + 2);
      }
      if (kk < 0 || kk >= g.nz) continue;
      cp_async16(st + (size_t)r * nx + 4 * q, dprev + ((size_t)kk * g.ny + jj) * nx + 4 * q);
    }
    const size_t r0 = (size_t)row * nx;
    float4 ro[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ro[q] = reinterpret_cast<const float4*>(rres + r0 + 2 * (t + q * T))[0];
    cp_async_wait_all();
    __syncthreads();
    const float2 ca = cff[k], cc = cff[g.nz + k], cd = cff[2 * g.nz + k];
    const float xh = to_real<float>(g.rdx2), xl = low_part(g.rdx2);
    const float yh = to_real<float>(g.rdy2), yl = low_part(g.rdy2);
    const bool up = k < g.nz - 1, dn = k > 0;
    const float* sc = st + (size_t)(line + 1) * nx;
    const float* sn = sc + nx;
    const float* ss = sc - nx;
    const float* sd = st + (size_t)(lines + 2 + line) * nx;
    const float* su = st + (size_t)(2 * lines + 2 + line) * nx;
    float2 val[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = 2 * (t + q * T);
      const float2 f = *reinterpret_cast<const float2*>(sc + i);
      const float2 fn = *reinterpret_cast<const float2*>(sn + i);
      const float2 fs = *reinterpret_cast<const float2*>(ss + i);
      const float2 fu = up ? *reinterpret_cast<const float2*>(su + i) : make_float2(0.f, 0.f);
      const float2 fd = dn ? *reinterpret_cast<const float2*>(sd + i) : make_float2(0.f, 0.f);
      const float4 o = resupd_pair(f, sc[wrap_prev(i, nx)], sc[wrap_add(i, 2, nx)], fn, fs, fu, fd, up, dn, ro[q],
                                   ca, cc, cd, xh, xl, yh, yl);
      if (stats) rr = fmaf(o.x, o.x, fmaf(o.z, o.z, rr));
      val[q] = make_float2(o.x, o.z);
      reinterpret_cast<float4*>(rres + r0 + i)[0] = o;
    }
    __syncthreads();  // the transform buffers lie over the staged rows
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[pad8(t + q * T)] = val[q];
  } else if (active) {
    const int nx = g.nx;
    k = row / g.ny;
    const size_t r0 = (size_t)row * nx;
    if (MODE == R32_FIRST) {
      // the thread's 8 points t + q T stay in registers for the first FFT pass
      const double2* s = reinterpret_cast<const double2*>(b + r0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = t + q * T;
        const double2 x = s[n];
        const float hx = to_real<float>(x.x), hy = to_real<float>(x.y);
        // row sum of b without FP64 arithmetic: TwoSum of the FP32 heads,
        // the tails and the rounding errors collected in fc
        two_sum_acc(fs, fc, hx);
        two_sum_acc(fs, fc, hy);
        fc = __fadd_rn(fc, __fadd_rn(low_part(x.x), low_part(x.y)));
        if (stats) {
          fs2 = fmaf(hx, hx, fmaf(hy, hy, fs2));
          const unsigned long long ax = (unsigned long long)__double_as_longlong(x.x) & 0x7fffffffffffffffull;
          const unsigned long long ay = (unsigned long long)__double_as_longlong(x.y) & 0x7fffffffffffffffull;
          amax = max(amax, max(ax, ay));
        }
        zr[q] = make_float2(hx, hy);
      }
    } else if (MODE == R32_RESID) {
      const int j = row - k * g.ny;
      const size_t NXY = (size_t)nx * g.ny;
      const size_t rjp = ((size_t)k * g.ny + (wrap_next(j, g.ny))) * nx;
      const size_t rjm = ((size_t)k * g.ny + (wrap_prev(j, g.ny))) * nx;
      const double pc = m.pc[k], pa = m.pa[k], pd = m.pdiag[k];
      const double mean = scal[S_BMEAN];
      const double ax = -g.rdx2, ay = -g.rdy2;
      const bool up = k < g.nz - 1, dn = k > 0;
      for (int n = t; n < M; n += T) {
        const int i = 2 * n;
        const double2 f = *reinterpret_cast<const double2*>(phi + r0 + i);
        const double fw = phi[r0 + (wrap_prev(i, nx))];
        const double fe = phi[r0 + (wrap_add(i, 2, nx))];
        const double2 fn = *reinterpret_cast<const double2*>(phi + rjp + i);
        const double2 fs = *reinterpret_cast<const double2*>(phi + rjm + i);
        const double2 bb = *reinterpret_cast<const double2*>(b + r0 + i);
        // r = (b - mean) + pdiag phi - rdx2 (phi_w + phi_e) - rdy2 (phi_s + phi_n)
        //     - pc phi_up - pa phi_down
        double rx = fma(pd, f.x, bb.x - mean);
        double ry = fma(pd, f.y, bb.y - mean);
        rx = fma(ax, fw + f.y, rx);
        ry = fma(ax, f.x + fe, ry);
        rx = fma(ay, fn.x + fs.x, rx);
        ry = fma(ay, fn.y + fs.y, ry);
        if (up) {
          const double2 fu = *reinterpret_cast<const double2*>(phi + r0 + NXY + i);
          rx = fma(-pc, fu.x, rx);
          ry = fma(-pc, fu.y, ry);
        }
        if (dn) {
          const double2 fd = *reinterpret_cast<const double2*>(phi + r0 - NXY + i);
          rx = fma(-pa, fd.x, rx);
          ry = fma(-pa, fd.y, ry);
        }
        const float2 r32 = make_float2(to_real<float>(rx), to_real<float>(ry));
        if (stats) rr = fmaf(r32.x, r32.x, fmaf(r32.y, r32.y, rr));
        buf[pad8(n)] = r32;
        reinterpret_cast<float4*>(rres + r0 + i)[0] = make_float4(r32.x, low_part(rx), r32.y, low_part(ry));
      }
    } else {  // R32_RESUPD
      const int j = row - k * g.ny;
      const size_t NXY = (size_t)nx * g.ny;
      const size_t rjp = ((size_t)k * g.ny + (wrap_next(j, g.ny))) * nx;
      const size_t rjm = ((size_t)k * g.ny + (wrap_prev(j, g.ny))) * nx;
      const float2 ca = cff[k], cc = cff[g.nz + k], cd = cff[2 * g.nz + k];
      const float xh = to_real<float>(g.rdx2), xl = low_part(g.rdx2);
      const float yh = to_real<float>(g.rdy2), yl = low_part(g.rdy2);
      const bool up = k < g.nz - 1, dn = k > 0;
      for (int n = t; n < M; n += T) {
        const int i = 2 * n;
        const float2 f = *reinterpret_cast<const float2*>(dprev + r0 + i);
        const float fw = dprev[r0 + (wrap_prev(i, nx))];
        const float fe = dprev[r0 + (wrap_add(i, 2, nx))];
        const float2 fn = *reinterpret_cast<const float2*>(dprev + rjp + i);
        const float2 fs = *reinterpret_cast<const float2*>(dprev + rjm + i);
        const float2 fu = up ? *reinterpret_cast<const float2*>(dprev + r0 + NXY + i) : make_float2(0.f, 0.f);
        const float2 fd = dn ? *reinterpret_cast<const float2*>(dprev + r0 - NXY + i) : make_float2(0.f, 0.f);
        const float4 ro = reinterpret_cast<const float4*>(rres + r0 + i)[0];
        const float4 o = resupd_pair(f, fw, fe, fn, fs, fu, fd, up, dn, ro, ca, cc, cd, xh, xl, yh, yl);
        if (stats) rr = fmaf(o.x, o.x, fmaf(o.z, o.z, rr));
        buf[pad8(n)] = make_float2(o.x, o.z);
        reinterpret_cast<float4*>(rres + r0 + i)[0] = o;
      }
    }
  }
  if (MODE == R32_FIRST) {
    if constexpr (GEN) fft_line_from_regs<false, true>(buf, M, zr, stw, 2, t, active);
    else fft_line_from_regs<false, false, true>(buf, M, zr, stp, 2, t, active);
  } else {
    __syncthreads();
    if constexpr (GEN) fft_line<false, true>(buf, M, stw, 2, t, active);
    else fft_line_pt<false>(buf, M, stp, t, active);
  }
  if (active) {
    float2* out = spec + (size_t)row * g.P;
    for (int q = t; q <= M / 2; q += T) {
      const float2 zk = buf[pad8(q)];
      if (q == 0) {
        out[0] = make_float2(zk.x + zk.y, 0.f);
        out[M] = make_float2(zk.x - zk.y, 0.f);
        continue;
      }
      const float2 zm = buf[pad8(M - q)];
      // FP32 arithmetic is not what limits this kernel: the halves stay as
      // multiplies (a halved table would cost every block its fill)
      const float2 E = make_float2((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
      const float2 O = make_float2((zk.y + zm.y) * 0.5f, (zm.x - zk.x) * 0.5f);
      const float2 wO = cmul(O, stw[q]);
      out[q] = cadd(E, wO);
      if (q != M / 2) out[M - q] = cconj(csub(E, wO));
    }
  }
  if (MODE == R32_FIRST) {
    const double s_row = to_double(fs) + to_double(fc);
    const double sw = active ? m.dzc[k] * s_row : 0.0;
    const double a = block_sum_d(sw, red);
    const double c = block_sum_d(s_row, red);
    const double d = stats ? block_sum_d(to_double(fs2), red) : 0.0;
    if (threadIdx.x == 0) {
      part[3 * blockIdx.x] = a;
      part[3 * blockIdx.x + 1] = c;
      part[3 * blockIdx.x + 2] = d;
    }
    if (stats) {
      for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((threadIdx.x & 31) == 0 && amax > 0ull)
        atomicMax(reinterpret_cast<unsigned long long*>(scal + S_RHS_ABSMAX), amax);
    }
  } else if (stats) {
    const double a = block_sum_d(to_double(rr), red);
    if (threadIdx.x == 0) part[3 * blockIdx.x] = a;
  }
}

// --------------------------------------------------------------------------
// Inverse x transform: X_k, k = 0..M -> nx reals (imaginary parts of X_0 and
// X_M are ignored). Z'_k = E'_k + i O'_k with E'_k = X_k + conj X_{M-k},
// O'_k = (X_k - conj X_{M-k}) conj(w_k); an inverse M-point FFT gives
// nx (x_2n + i x_2n+1) before the 1/(nx ny) normalisation `scale`.
// MODE 0 writes phi = scale * x (FP64 path). Mixed precision, with per-block
// partials part[2 blk] = ||delta||^2 (FP32 per thread) and part[2 blk + 1] =
// sum dzc * delta (FP32 per thread, compensated in MODE 2):
//   MODE 2 writes phi = delta (the first correction);
//   MODE 1 adds phi += delta - mean_W(phi) (the mean measured after the
//   previous correction), so that the gauge of phi is kept as it is refined.
// TAN: as in k_r2c_x, with the inverse tables.
template <typename R, int MODE, bool GEN, bool TAN = false>
__global__ void __launch_bounds__(512, TAN ? 2 : 0) k_c2r_x(Grid g, Metric m,
                                               const typename cplx<R>::T* __restrict__ spec,
                                               const typename cplx<R>::T* __restrict__ tw,
                                               double scale, double* __restrict__ phi,
                                               const double* __restrict__ skip,
                                               double* __restrict__ part,
                                               const double* __restrict__ pmean,
                                               float* __restrict__ dprev,
                                               const double* __restrict__ ttab, int tlen) {
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
  C* stw = sm + lines * stride;  // twiddle table, nx entries
  C* stp = stw + g.nx;           // per-pass tables of the M-point FFT (power-of-two M)
  C* stq = stp + (TAN ? max(M, (tlen + 1) / 2) : M);  // MODE 0: packing twiddles scale * w_k, k <= M/2
  for (int q = threadIdx.x; q < g.nx; q += blockDim.x) stw[q] = tw[q];
  if constexpr (TAN) {
    double* sd = reinterpret_cast<double*>(stp);
    for (int q = threadIdx.x; q < tlen; q += blockDim.x) sd[q] = ttab[q];
  } else if (!GEN) {
    pass_twiddles(stp, tw, M, 2, threadIdx.x, blockDim.x);
  }
  if (MODE == 0)
    for (int q = threadIdx.x; q <= M / 2; q += blockDim.x) stq[q] = cscale(tw[q], (R)scale);
  if (active) {
    const C* in = spec + (size_t)row * g.P;
    for (int k = t; k <= M; k += T) buf[pad8(k)] = in[k];
  }
  __syncthreads();
  if (active) {
    for (int k = t; k <= M / 2; k += T) {
      if (k == 0) {
        const R x0 = buf[pad8(0)].x, xm = buf[pad8(M)].x;
        buf[pad8(0)] = MODE == 0 ? C{(x0 + xm) * (R)scale, (x0 - xm) * (R)scale} : C{x0 + xm, x0 - xm};
        continue;
      }
      const C a = buf[pad8(k)], b = buf[pad8(M - k)];
      const C E = C{a.x + b.x, a.y - b.y};
      // Z'_k = E + i O ; Z'_{M-k} = conj(E) + i conj(O). MODE 0 applies the
      // normalisation here (the transform is linear): O from the scaled
      // table, E through the FMAs, so the output needs no multiply.
      if (MODE == 0) {
        const R sc = (R)scale;
        const C O = cmulc(C{a.x - b.x, a.y + b.y}, stq[k]);
        buf[pad8(k)] = C{fma(sc, E.x, -O.y), fma(sc, E.y, O.x)};
        if (k != M / 2) buf[pad8(M - k)] = C{fma(sc, E.x, O.y), fma(-sc, E.y, O.x)};
      } else {
        const C O = cmulc(C{a.x - b.x, a.y + b.y}, stw[k]);
        buf[pad8(k)] = C{E.x - O.y, E.y + O.x};
        if (k != M / 2) buf[pad8(M - k)] = C{E.x + O.y, O.x - E.y};
      }
    }
  }
  __syncthreads();
  // FP32 lines of power-of-two length keep the last FFT pass in registers:
  // its outputs are the thread's points t + q T written out below
  constexpr bool REGS = !GEN && std::is_same<R, float>::value;
  C zr[8];
  if constexpr (REGS) fft_line_pow2_to_regs<true, true>(buf, M, zr, stp, 2, t, active);
  else if constexpr (GEN) fft_line<true, true>(buf, M, stw, 2, t, active);
  else if constexpr (TAN)  // launched for FP64 lines only (the cast is the identity there)
    fft_line_tan_ix<true>(reinterpret_cast<double2*>(buf), M, reinterpret_cast<const double*>(stp), t, active, PadIx{});
  else fft_line_pt<true>(buf, M, stp, t, active);
  R d2 = (R)0, dsum = (R)0, dcomp = (R)0;
  double psum = 0.0;
  if (active) {
    double2* o2 = reinterpret_cast<double2*>(phi + (size_t)row * g.nx);
    const R sc = (R)scale;
    // MODE 1 removes the weighted mean of phi measured after the previous
    // correction (rounded to the working precision) while adding this one
    const R pm = MODE == 1 ? to_real<R>(*pmean) : (R)0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int n = t + q * T;
      const C z = REGS ? zr[q] : buf[pad8(n)];
      if (MODE == 0) {
        o2[n] = make_double2((double)z.x, (double)z.y);  // normalised in the packing
      } else {
        // rounded products (no contraction into the sums below): the sums
        // must see exactly the values stored in phi
        const R dx = mul_rn(z.x, sc), dy = mul_rn(z.y, sc);
        d2 += dx * dx + dy * dy;
        if (MODE == 1) {        // later corrections are small: their sum in FP32
          const R ex = dx - pm, ey = dy - pm;
          double2 r = make_double2(to_double(ex), to_double(ey));
          const double2 old = o2[n];
          r.x += old.x;
          r.y += old.y;
          o2[n] = r;
          dsum += dx + dy;
          // the correction as added, for the next residual update
          if (dprev) reinterpret_cast<typename cplx<R>::T*>(dprev + (size_t)row * g.nx)[n] =
              typename cplx<R>::T{ex, ey};
        } else {                // the first correction is the bulk of phi:
          o2[n] = make_double2(to_double(dx), to_double(dy));
          // compensated FP32 sum: exact rounding error of every addition
          // (TwoSum) collected in dcomp
          two_sum_acc(dsum, dcomp, dx);
          two_sum_acc(dsum, dcomp, dy);
        }
      }
    }
    if (MODE == 1) psum = to_double(dsum) * m.dzc[row / g.ny];
    if (MODE == 2) psum = (to_double(dsum) + to_double(dcomp)) * m.dzc[row / g.ny];
  }
  if (MODE != 0) {
    // per-block ||delta||^2 and sum of dzc * phi (weighted mean of phi)
    __shared__ double red[512];
    const double a = block_sum_d(to_double(d2), red);
    const double b = block_sum_d(psum, red);
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
  }
}

// --------------------------------------------------------------------------
// Complex FFT along y for a tile of TK consecutive kx columns of one z plane.
// TAN (FP64, power-of-two ny >= 64): the radix-8 passes with their twiddles in
// tangent form (stockham_pass8_tan), `ttab` the direction's tables of
// tan_tables, `tlen` doubles; otherwise the twiddles come from `tw`.
template <typename R, bool INV, int TK, bool GEN, bool TAN = false>
__global__ void __launch_bounds__(1024) k_fft_y(Grid g, typename cplx<R>::T* __restrict__ spec,
                                                const typename cplx<R>::T* __restrict__ tw,
                                                const double* __restrict__ skip,
                                                const double* __restrict__ ttab = nullptr, int tlen = 0) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int Ny = g.ny, T = Ny / 8;
  const int z = blockIdx.y, kx0 = blockIdx.x * TK;
  const int ncol = min(TK, g.M + 1 - kx0);
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int stride = pad8(Ny) + 1;
  C* stw = sm + TK * stride;  // twiddle table, ny entries (TAN: the tangent tables)
  if constexpr (TAN) {
    double* st = reinterpret_cast<double*>(stw);
    for (int q = threadIdx.x; q < tlen; q += blockDim.x) st[q] = ttab[q];
  } else {
    for (int q = threadIdx.x; q < Ny; q += blockDim.x) stw[q] = tw[q];
  }
  C* base = spec + (size_t)z * Ny * g.P + kx0;
  // Ny * TK = 8 * blockDim.x: eight independent loads per thread, all in flight
  C vals[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    const int ky = e / TK, c = e - (e / TK) * TK;
    if (c < ncol) vals[q] = base[(size_t)ky * g.P + c];
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    const int ky = e / TK, c = e - (e / TK) * TK;
    if (c < ncol) sm[c * stride + pad8(ky)] = vals[q];
  }
  __syncthreads();
  if constexpr (TAN)
    fft_line_tan_ix<INV>(sm + line * stride, Ny, reinterpret_cast<const double*>(stw), t, line < ncol, PadIx{});
  else
    fft_line<INV, GEN>(sm + line * stride, Ny, stw, 1, t, line < ncol);
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
// Forward elimination and back substitution of one column (rows k = 0..nz-1,
// pa[0] = 0), with the loads of the next U rows issued together so that the
// memory latency is paid once per U rows rather than once per row.
template <typename R, typename C>
__device__ __forceinline__ void thomas_column(C* __restrict__ col, const R* __restrict__ mt,
                                              const R* __restrict__ pa, const R* __restrict__ pc,
                                              int nz, size_t plane, size_t tplane) {
  // rows loaded U at a time before they are used (the loads of a batch in
  // flight together; a store to the column and the next row's load cannot be
  // reordered by the compiler): 8 rows in FP32, 4 in FP64 (registers)
  constexpr int U = sizeof(R) == 8 ? 4 : 8;
  C dv[U];
  R mv[U];
  C dp = C{(R)0, (R)0};
  for (int kb = 0; kb < nz; kb += U) {
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = kb + q;
      if (k < nz) {
        dv[q] = col[k * plane];
        mv[q] = mt[k * tplane];
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = kb + q;
      if (k < nz) {
        const R ak = pa[k];
        dp = C{(dv[q].x - ak * dp.x) * mv[q], (dv[q].y - ak * dp.y) * mv[q]};
        col[k * plane] = dp;
      }
    }
  }
  C x = dp;
  for (int kb = nz - 2; kb >= 0; kb -= U) {
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = kb - q;
      if (k >= 0) {
        dv[q] = col[k * plane];
        mv[q] = mt[k * tplane];
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int k = kb - q;
      if (k >= 0) {
        const R cp = pc[k] * mv[q];
        x = C{dv[q].x - cp * x.x, dv[q].y - cp * x.y};
        col[k * plane] = x;
      }
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(128) k_thomas(Grid g, Metric m, typename cplx<R>::T* __restrict__ spec,
                                                const R* __restrict__ mtab,
                                                const R* __restrict__ pa, const R* __restrict__ pc,
                                                const double* __restrict__ lamx,
                                                const double* __restrict__ lamy, double lam_thr,
                                                const double* __restrict__ skip) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  // one system per thread over the flattened (ky, kx) index: consecutive
  // threads take consecutive kx of a row and continue on the next row, so no
  // block is left with the lone kx = M column of a row (every FP64 warp
  // instruction costs the same issue time however few lanes are active)
  const int W = g.M + 1;
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (sidx >= g.ny * W) return;
  const int ky = sidx / W, kx = sidx - ky * W;
  if (kx == 0 && ky == 0) return;
  const int kyh = min(ky, g.ny - ky);
  if (lam_thr > 0.0 && lamx[kx] + lamy[kyh] < lam_thr) return;
  const size_t plane = (size_t)g.ny * g.P;
  const size_t tplane = (size_t)g.nyh * W;
  C* col = spec + (size_t)ky * g.P + kx;
  const R* mt = mtab + (size_t)kyh * W + kx;
  thomas_column<R, C>(col, mt, pa, pc, g.nz, plane, tplane);
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
  const int W = g.M + 1;
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;  // flattened (ky, kx), as in k_thomas
  if (sidx >= g.ny * W) return;
  const int ky = sidx / W, kx = sidx - ky * W;
  if (kx == 0 && ky == 0) return;
  const int kyh = min(ky, g.ny - ky);
  const size_t plane = (size_t)g.ny * g.P;
  const size_t tplane = (size_t)g.nyh * W;
  float2* col = spec + (size_t)ky * g.P + kx;
  const int nz = g.nz;
  if (lowslot[(size_t)ky * W + kx] >= 0) return;  // FP64 warp solver (k_tridiag_warp)
  const float* mt = mtab32 + (size_t)kyh * W + kx;
  thomas_column<float, float2>(col, mt, pa32, pc32, nz, plane, tplane);
}

// --------------------------------------------------------------------------
// Warp-partitioned FP64 solve of one tridiagonal system per warp (the
// parallel-cyclic-reduction variant for long columns / few systems): rows
// a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k with the Poisson coefficients
// a = pa, c = pc, b = -pa - pc - lambda, complex d, k = 0..nz-1.
//   1. lane l owns rows [s_l, e_l); with its last unknown X_l = x_{e_l - 1}
//      and X_{l-1} treated as known, its interior rows s_l..e_l-2 are solved
//      by Thomas for three right-hand sides, x_r = g_r + al_r X_{l-1} + be_r X_l;
//   2. the last row of each chunk gives one equation in X_{l-1}, X_l, X_{l+1}
//      (the next lane's first interior row arrives by shuffle): a 32-unknown
//      tridiagonal system, solved by parallel cyclic reduction over shuffles;
//   3. each lane reconstructs its interior rows.
// Used for the nearly singular low modes of the mixed-precision solve: the
// data column is FP32, the elimination FP64. Scratch: 4 doubles per interior
// row per lane in shared memory.
__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_up_d(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_dn_d(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

__host__ __device__ inline int warp_rows(int nz) { return nz < 64 ? 2 : (nz + 31) / 32; }
// warps per block so that the per-lane scratch (5 doubles per row) stays <= 160 KB
inline int warps_per_block(int nz) {
  const size_t per_warp = (size_t)32 * 5 * warp_rows(nz) * sizeof(double);
  int w = (int)((160u << 10) / per_warp);
  return w < 1 ? 1 : (w > 4 ? 4 : w);
}

template <typename CT>
__global__ void __launch_bounds__(128) k_tridiag_warp(Grid g, Metric m, CT* __restrict__ spec,
                                                      const int2* __restrict__ modes, int nmodes,
                                                      const double* __restrict__ lamx,
                                                      const double* __restrict__ lamy,
                                                      const double* __restrict__ skip) {
  using R = decltype(CT::x);
  if (skip && *skip != 0.0) return;
  extern __shared__ double wsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mi = blockIdx.x * (blockDim.x >> 5) + warp;
  // modes == nullptr: every (ky, kx) by index, the singular (0,0) excluded
  bool have = mi < nmodes;  // warp-uniform
  const int nz = g.nz;
  const int L = warp_rows(nz);             // rows per lane (>= 2)
  const int lanes = (nz + L - 1) / L;      // lanes that own rows (<= 32)
  const int s = lane * L;
  const int e = lane < lanes ? min(s + L, nz) : s;
  double* sg = wsm + (size_t)threadIdx.x * 5 * L;  // per row: g.x, g.y, al, be, c'
  int ky = 0, kx = 0;
  if (have) {
    if (modes) {
      const int2 md = modes[mi];
      ky = md.x;
      kx = md.y;
    } else {
      ky = mi / (g.M + 1);
      kx = mi - ky * (g.M + 1);
    }
  }
  have = have && !(kx == 0 && ky == 0);
  const bool used = have && lane < lanes;  // owns rows s..e-1 (at least one)
  const int n_int = used ? e - s - 1 : 0;  // interior rows s..e-2
  const double lam = have ? lamx[kx] + lamy[min(ky, g.ny - ky)] : 0.0;
  const size_t plane = (size_t)g.ny * g.P;
  CT* col = spec + (size_t)ky * g.P + kx;
  // ---- 1. Thomas on the interior rows with right-hand sides d, -a_s e_first, -c e_last
  {
    double cprev = 0.0, gx = 0.0, gy = 0.0, al = 0.0, be = 0.0;
    for (int q = 0; q < n_int; ++q) {
      const int r = s + q;
      const bool last = q == n_int - 1;
      const double a = m.pa[r];  // a * (previous) vanishes at q = 0: all accumulators are 0
      const double b = -m.pa[r] - m.pc[r] - lam;
      const double rinv = 1.0 / (b - a * cprev);
      const CT d = col[(size_t)r * plane];
      gx = ((double)d.x - a * gx) * rinv;
      gy = ((double)d.y - a * gy) * rinv;
      al = ((q == 0 ? -m.pa[s] : 0.0) - a * al) * rinv;
      be = ((last ? -m.pc[r] : 0.0) - a * be) * rinv;
      cprev = last ? 0.0 : m.pc[r] * rinv;
      double* o = sg + 5 * q;
      o[0] = gx;
      o[1] = gy;
      o[2] = al;
      o[3] = be;
      o[4] = cprev;
    }
    for (int q = n_int - 2; q >= 0; --q) {
      double* o = sg + 5 * q;
      const double* n = o + 5;
      const double cp = o[4];
      o[0] -= cp * n[0];
      o[1] -= cp * n[1];
      o[2] -= cp * n[2];
      o[3] -= cp * n[3];
    }
  }
  // first interior row of this lane, needed by the previous lane
  double fgx = 0.0, fgy = 0.0, fal = 0.0, fbe = 0.0;
  if (n_int > 0) {
    fgx = sg[0];
    fgy = sg[1];
    fal = sg[2];
    fbe = sg[3];
  }
  const double ngx = shfl_dn_d(fgx, 1), ngy = shfl_dn_d(fgy, 1);
  const double nal = shfl_dn_d(fal, 1), nbe = shfl_dn_d(fbe, 1);
  const int nn_int = __shfl_down_sync(0xffffffffu, n_int, 1);
  // ---- 2. interface equation of row e-1: A X_{l-1} + B X_l + C X_{l+1} = D
  double A = 0.0, B = 1.0, C = 0.0, Dx = 0.0, Dy = 0.0;
  if (used) {
    const int r = e - 1;
    const double a = m.pa[r], c = m.pc[r];
    const CT d = col[(size_t)r * plane];
    Dx = (double)d.x;
    Dy = (double)d.y;
    B = -m.pa[r] - m.pc[r] - lam;
    if (n_int > 0) {  // x_{e-2} = g + al X_{l-1} + be X_l
      const double* o = sg + 5 * (n_int - 1);
      A = a * o[2];
      B += a * o[3];
      Dx -= a * o[0];
      Dy -= a * o[1];
    } else {
      A = a;
    }
    if (lane + 1 < lanes) {  // x_e = next lane's first row
      if (nn_int > 0) {       // = g' + al' X_l + be' X_{l+1}
        B += c * nal;
        C = c * nbe;
        Dx -= c * ngx;
        Dy -= c * ngy;
      } else {
        C = c;
      }
    }
  }
  // parallel cyclic reduction of the lane system (unused lanes: identity rows)
  for (int st = 1; st < 32; st <<= 1) {
    const double Am = shfl_up_d(A, st), Bm = shfl_up_d(B, st), Cm = shfl_up_d(C, st);
    const double Dxm = shfl_up_d(Dx, st), Dym = shfl_up_d(Dy, st);
    const double Ap = shfl_dn_d(A, st), Bp = shfl_dn_d(B, st), Cp = shfl_dn_d(C, st);
    const double Dxp = shfl_dn_d(Dx, st), Dyp = shfl_dn_d(Dy, st);
    const bool lo = lane >= st, hi = lane + st < 32;
    const double k1 = lo ? A / Bm : 0.0;
    const double k2 = hi ? C / Bp : 0.0;
    const double nA = lo ? -Am * k1 : 0.0;
    const double nC = hi ? -Cp * k2 : 0.0;
    B = B - (lo ? Cm * k1 : 0.0) - (hi ? Ap * k2 : 0.0);
    Dx = Dx - (lo ? Dxm * k1 : 0.0) - (hi ? Dxp * k2 : 0.0);
    Dy = Dy - (lo ? Dym * k1 : 0.0) - (hi ? Dyp * k2 : 0.0);
    A = nA;
    C = nC;
  }
  const double Xx = Dx / B, Xy = Dy / B;
  double Xmx = shfl_up_d(Xx, 1), Xmy = shfl_up_d(Xy, 1);
  if (lane == 0) {
    Xmx = 0.0;
    Xmy = 0.0;
  }
  // ---- 3. reconstruct the interior rows, write the FP32 column
  if (used) {
    for (int q = 0; q < n_int; ++q) {
      const double* o = sg + 5 * q;
      const double vx = o[0] + o[2] * Xmx + o[3] * Xx;
      const double vy = o[1] + o[2] * Xmy + o[3] * Xy;
      col[(size_t)(s + q) * plane] = CT{(R)vx, (R)vy};
    }
    col[(size_t)(e - 1) * plane] = CT{(R)Xx, (R)Xy};
  }
}

// --------------------------------------------------------------------------
// Exact solution of the singular (0,0) mode in FP64 (one block): remove the
// dzc-weighted mean of bhat (solvability), flux prefix sums
// F_{k+1} = F_k + dzc_k bhat_k, phi_k = phi_{k-1} + dzf_k F_k, then the gauge
// (zero dzc-weighted mean). Also records the removed mean of the rhs.
// Thread t owns the rows [t E, t E + E); the two recurrences are prefix sums,
// taken as block-wide exclusive scans of the per-thread partial sums.

// Exclusive prefix sum over the block of one double per thread, and the block
// total. ws: 32 doubles of shared scratch; every thread of the block calls it.
__device__ __forceinline__ double block_excl_scan(double v, double* ws, double* total) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  double ex = __shfl_up_sync(FULL, x, 1);
  if (lane == 0) ex = 0.0;
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;  // inclusive over the warps
  }
  __syncthreads();
  const double before = warp > 0 ? ws[warp - 1] + ex : ex;
  *total = ws[nw - 1];
  __syncthreads();  // ws free for the next call
  return before;
}

// The (0,0)-mode solve on the nz values zb[0..nz) (shared memory, doubles),
// in place: zb becomes phi - mean_W(phi). ws: 32 doubles of shared scratch.
// Every thread of the block calls it.
__device__ __forceinline__ void zero_mode_column(const Grid& g, const Metric& m, double* zb, double* ws,
                                                 double* scal) {
  const int nz = g.nz;
  const int E = (nz + blockDim.x - 1) / blockDim.x;
  const int k0 = min((int)threadIdx.x * E, nz), k1 = min(k0 + E, nz);
  const double* __restrict__ dzc = m.dzc;
  const double* __restrict__ dzf = m.dzf;
  double sw = 0.0, sb = 0.0;
  for (int k = k0; k < k1; ++k) {
    sw += dzc[k];
    sb += dzc[k] * zb[k];
  }
  double tsw, tsb, unused;
  block_excl_scan(sw, ws, &tsw);
  block_excl_scan(sb, ws, &tsb);
  const double mu = tsb / tsw;
  if (threadIdx.x == 0) scal[S_RHS_MEAN] = mu / ((double)g.nx * (double)g.ny);
  // F at the first owned row: sum over all earlier rows of dzc (b - mu)
  double f = 0.0;
  for (int k = k0; k < k1; ++k) f += dzc[k] * (zb[k] - mu);
  const double F0 = block_excl_scan(f, ws, &unused);
  // phi at the row before the first owned one: sum of dzf_j F_j, 1 <= j < k0
  double gs = 0.0, Fk = F0;
  for (int k = k0; k < k1; ++k) {
    if (k > 0) gs += dzf[k] * Fk;
    Fk += dzc[k] * (zb[k] - mu);
  }
  double ph = block_excl_scan(gs, ws, &unused);
  double sp = 0.0;
  Fk = F0;
  for (int k = k0; k < k1; ++k) {
    if (k > 0) ph += dzf[k] * Fk;
    Fk += dzc[k] * (zb[k] - mu);
    zb[k] = ph;
    sp += dzc[k] * ph;
  }
  double tsp;
  block_excl_scan(sp, ws, &tsp);
  const double pm = tsp / tsw;
  for (int k = k0; k < k1; ++k) zb[k] -= pm;
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(1024) k_zero_mode(Grid g, Metric m, typename cplx<R>::T* __restrict__ spec,
                                                    double* scal, const double* __restrict__ skip) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ double zb[];  // nz values, then 32 doubles of scan scratch
  const int nz = g.nz;
  const size_t plane = (size_t)g.ny * g.P;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) zb[k] = (double)spec[k * plane].x;
  __syncthreads();
  zero_mode_column(g, m, zb, zb + nz, scal);
  for (int k = threadIdx.x; k < nz; k += blockDim.x) spec[k * plane] = C{(R)zb[k], (R)0};
}

// --------------------------------------------------------------------------
// Mixed precision, small nz: the forward y transform, the wall-normal solves
// and the inverse y transform of one kx column in one kernel (the FFT-Thomas-
// FFT sequence of Sec. 2.2 on a brick that stays in shared memory). One block
// per kx holds the brick [nz][ny] of that column (rows of pad8(ny) + 1
// slots), the column's FP32 pivots [nz][ny/2 + 1] (the table transposed to
// [kx][k][kyh], one contiguous slice) and, for the column's low modes, their
// FP64 pivots and FP64 d'. It gathers the brick, transforms its nz lines
// along y, solves the ny wall-normal systems of the column with every operand
// and the intermediate d' on chip -- FP32 Thomas for most modes, FP64 Thomas
// with the FP64 table for the low modes (lowslot >= 0), the exact FP64 prefix
// sums for (0,0) in block kx = 0 -- transforms back and scatters the column.
// The arithmetic per mode is that of k_fft_y / k_thomas_mixed / k_zero_mode;
// the low modes take the table-based FP64 Thomas sweep instead of the
// warp-partitioned one. Taken when all of it fits in shared memory and the
// FP32 spectral array fits in half the L2 (there the separate passes are
// bound by latency rather than by HBM, and the column gathers, 8 of every 32
// bytes of a sector, are served from L2), by default only for nz ny <= 8192
// and ny <= 512: with one block of up to 227 KB per SM the kernel is itself
// latency-bound, and on GB300 it beats the separate passes only on small
// bricks (measured 1.4-2.1x there, 10% slower at 512 x 512 x 32).
struct YtLayout {
  size_t brick, tw, piv, lowpiv, lowd, zb, total;  // byte offsets
};
__host__ __device__ inline YtLayout yt_layout(const Grid& g, int lmax) {
  // every region starts on a 16-byte boundary (double2 and float2 accesses)
  auto up16 = [](size_t b) { return (b + 15) / 16 * 16; };
  YtLayout L;
  size_t o = 0;
  L.brick = o;
  o += up16((size_t)g.nz * (pad8(g.ny) + 1) * sizeof(float2));
  L.tw = o;
  o += up16((size_t)g.ny * sizeof(float2));
  L.piv = o;
  o += up16((size_t)g.nz * g.nyh * sizeof(float));
  L.lowpiv = o;
  o += up16((size_t)lmax * g.nz * sizeof(double));
  L.lowd = o;
  o += up16((size_t)lmax * g.nz * sizeof(double2));
  L.zb = o;
  o += up16((size_t)(g.nz + 32) * sizeof(double));
  L.total = o;
  return L;
}

template <bool GEN>
__global__ void __launch_bounds__(512) k_yfft_thomas32(Grid g, Metric m, float2* __restrict__ spec,
                                                       const float2* __restrict__ tw,
                                                       const float* __restrict__ mtabt32,
                                                       const double* __restrict__ mtab64,
                                                       const float* __restrict__ pa32,
                                                       const float* __restrict__ pc32,
                                                       const int* __restrict__ lowslot, int lmax,
                                                       double* scal, const double* __restrict__ skip) {
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(16) unsigned char yt_raw[];
  __shared__ int nlow_here;
  const int N = g.ny, nz = g.nz, W = g.M + 1, kx = blockIdx.x, nyh = g.nyh;
  const int LS = pad8(N) + 1;
  const YtLayout L = yt_layout(g, lmax);
  float2* brick = reinterpret_cast<float2*>(yt_raw + L.brick);
  float2* stw = reinterpret_cast<float2*>(yt_raw + L.tw);
  float* piv = reinterpret_cast<float*>(yt_raw + L.piv);           // [nz][nyh]
  double* lpiv = reinterpret_cast<double*>(yt_raw + L.lowpiv);     // [lmax][nz]
  double2* ld = reinterpret_cast<double2*>(yt_raw + L.lowd);       // [lmax][nz]
  double* zb = reinterpret_cast<double*>(yt_raw + L.zb);           // (0,0) column + 32 scratch
  const int tid = threadIdx.x, nth = blockDim.x;
  const size_t P = g.P;
  if (tid == 0) nlow_here = 0;
  // 1. gather the column (sixteen loads in flight per thread), the twiddles and
  //    the column's FP32 pivots
  const int tot = nz * N;
  for (int i0 = tid; i0 < tot; i0 += 16 * nth) {
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = i0 + q * nth;
      if (i < tot) {
        const int z = i / N, y = i - z * N;
        v[q] = spec[((size_t)z * N + y) * P + kx];
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = i0 + q * nth;
      if (i < tot) {
        const int z = i / N, y = i - z * N;
        brick[(size_t)z * LS + pad8(y)] = v[q];
      }
    }
  }
  for (int q = tid; q < N; q += nth) stw[q] = tw[q];
  const float* pslice = mtabt32 + (size_t)kx * nz * nyh;
  for (int q = tid; q < nz * nyh; q += nth) piv[q] = pslice[q];
  __syncthreads();
  // 2. forward transforms of the nz lines, N/8 threads per line
  const int T = N / 8, lpr = nth / T;
  for (int z0 = 0; z0 < nz; z0 += lpr) {
    const int z = z0 + tid / T;
    const bool act = tid < lpr * T && z < nz;
    fft_line<false, GEN>(brick + (size_t)(act ? z : 0) * LS, N, stw, 1, tid % T, act);
  }
  // 3. wall-normal solves, one ky per thread
  for (int ky = tid; ky < N; ky += nth) {
    if (kx == 0 && ky == 0) continue;  // exact prefix sums below
    const int kyh = min(ky, N - ky);
    float2* col = brick + pad8(ky);
    if (lowslot[(size_t)ky * W + kx] >= 0) {
      // nearly singular low mode: FP64 sweep with the FP64 pivot table; its
      // pivots are first copied to shared memory (independent loads), its d'
      // kept there in FP64
      const int j = atomicAdd(&nlow_here, 1);  // < lmax (the column's low-mode count)
      double* mp = lpiv + (size_t)j * nz;
      double2* dcol = ld + (size_t)j * nz;
      const double* mt = mtab64 + (size_t)kyh * W + kx;
      const size_t tplane = (size_t)nyh * W;
      for (int k = 0; k < nz; ++k) mp[k] = mt[k * tplane];
      double dx = 0.0, dy = 0.0;
      for (int k = 0; k < nz; ++k) {
        const float2 d = col[(size_t)k * LS];
        const double mk = mp[k], ak = m.pa[k];
        dx = ((double)d.x - ak * dx) * mk;
        dy = ((double)d.y - ak * dy) * mk;
        dcol[k] = make_double2(dx, dy);
      }
      col[(size_t)(nz - 1) * LS] = make_float2((float)dx, (float)dy);
      for (int k = nz - 2; k >= 0; --k) {
        const double2 e = dcol[k];
        const double cp = m.pc[k] * mp[k];
        dx = e.x - cp * dx;
        dy = e.y - cp * dy;
        col[(size_t)k * LS] = make_float2((float)dx, (float)dy);
      }
      continue;
    }
    // FP32 sweeps in blocks of U rows: the U loads of a block are issued
    // together, then the recurrence runs on registers (the per-row arithmetic
    // of thomas_column)
    constexpr int U = 8;
    const float* mt = piv + kyh;
    float2 dv[U];
    float mv[U];
    float2 dp = make_float2(0.f, 0.f);
    for (int kb = 0; kb < nz; kb += U) {
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = kb + q;
        if (k < nz) {
          dv[q] = col[(size_t)k * LS];
          mv[q] = mt[(size_t)k * nyh];
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = kb + q;
        if (k < nz) {
          const float ak = pa32[k];
          dp = make_float2((dv[q].x - ak * dp.x) * mv[q], (dv[q].y - ak * dp.y) * mv[q]);
          dv[q] = dp;
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = kb + q;
        if (k < nz) col[(size_t)k * LS] = dv[q];
      }
    }
    float2 x = dp;
    for (int kb = nz - 2; kb >= 0; kb -= U) {
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = kb - q;
        if (k >= 0) {
          dv[q] = col[(size_t)k * LS];
          mv[q] = mt[(size_t)k * nyh];
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = kb - q;
        if (k >= 0) {
          const float cp = pc32[k] * mv[q];
          x = make_float2(dv[q].x - cp * x.x, dv[q].y - cp * x.y);
          dv[q] = x;
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = kb - q;
        if (k >= 0) col[(size_t)k * LS] = dv[q];
      }
    }
  }
  __syncthreads();
  // 4. the singular (0,0) mode (block-uniform branch)
  if (kx == 0) {
    for (int k = tid; k < nz; k += nth) zb[k] = (double)brick[(size_t)k * LS].x;
    __syncthreads();
    zero_mode_column(g, m, zb, zb + nz, scal);
    for (int k = tid; k < nz; k += nth) brick[(size_t)k * LS] = make_float2((float)zb[k], 0.f);
    __syncthreads();
  }
  // 5. inverse transforms
  for (int z0 = 0; z0 < nz; z0 += lpr) {
    const int z = z0 + tid / T;
    const bool act = tid < lpr * T && z < nz;
    fft_line<true, GEN>(brick + (size_t)(act ? z : 0) * LS, N, stw, 1, tid % T, act);
  }
  // 6. scatter the column
  for (int i = tid; i < tot; i += nth) {
    const int z = i / N, y = i - z * N;
    spec[((size_t)z * N + y) * P + kx] = brick[(size_t)z * LS + pad8(y)];
  }
}

// Shared memory of the fused small-nz kernel for a column low-mode count lmax.
size_t yfft_thomas32_smem(const Grid& g, int lmax) { return yt_layout(g, lmax).total; }

cudaError_t init_yfft_thomas32(afid_ctx* c, int lmax) {
  c->fuse_yt = 0;
  const Grid& g = c->g;
  if (c->prec != AFID_MIXED || (c->flags & AFID_NO_FUSE) || g.ny < 8) return cudaSuccess;
  // by default only where it was measured faster than the separate passes
  if (!(c->flags & AFID_FUSE_SMALL_NZ) && ((long long)g.nz * g.ny > 8192 || g.ny > 512)) return cudaSuccess;
  int smem_optin = 0, l2 = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
  const size_t sm = yfft_thomas32_smem(g, lmax);
  const size_t spec_bytes = (size_t)g.nz * g.ny * g.P * sizeof(float2);
  // + the kernel's static shared memory (one int)
  if (sm + 64 > (size_t)smem_optin || spec_bytes > (size_t)l2 / 2) return cudaSuccess;
  const bool gen = !is_pow2(g.ny);
  cudaError_t e = cudaFuncSetAttribute(gen ? k_yfft_thomas32<true> : k_yfft_thomas32<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) {
    cudaGetLastError();
    return cudaSuccess;
  }
  c->yt_smem = sm;
  c->yt_lmax = lmax;
  c->yt_threads = yfft_thomas32_threads(g);
  c->fuse_yt = 1;
  return cudaSuccess;
}

int yfft_thomas32_threads(const Grid& g) {
  const int T = g.ny / 8;
  long long want = (long long)T * g.nz;
  if (want < g.ny) want = g.ny;
  want = (want + 31) / 32 * 32;
  return want > 512 ? 512 : (int)want;
}

static void launch_zero_mode_threads(const Grid& g, int* thr, size_t* sm) {
  int t = ((g.nz + 31) / 32) * 32;
  *thr = t > 1024 ? 1024 : t;
  *sm = (size_t)(g.nz + 32) * sizeof(double);
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
  if constexpr (sizeof(R) == sizeof(float))
    if (c->tma_y) return run_fft_y_tma<float>(c, tw, inv, skip);
  const Grid& g = c->g;
  const size_t ls = line_smem<R>(g.ny);
  // widest tile that keeps a block within 1024 threads and ~112 KB of shared memory
  int tk = 8;
  while (tk > 1 && ((size_t)tk * ls > 112 * 1024 || tk * (g.ny / 8) > 1024)) tk /= 2;
  dim3 grd(ceil_div(g.M + 1, tk), g.nz);
  const int thr = tk * (g.ny / 8);
  const bool gen = !is_pow2(g.ny);  // radix-3/5 passes needed
  if constexpr (sizeof(R) == sizeof(double)) {
    if (c->ytan64[0]) {  // tangent-form twiddles (power-of-two ny >= 64)
      const size_t sm = (size_t)tk * ls + (size_t)c->ytan_len * sizeof(double);
      const double* tt = c->ytan64[inv ? 1 : 0];
#define AFID_FFTYT(TKV)                                                                         \
  do {                                                                                          \
    auto kf = inv ? k_fft_y<double, true, TKV, false, true> : k_fft_y<double, false, TKV, false, true>; \
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);             \
    kf<<<grd, thr, sm, c->stream>>>(g, spec, tw, skip, tt, c->ytan_len);                        \
  } while (0)
      switch (tk) {
        case 8: AFID_FFTYT(8); break;
        case 4: AFID_FFTYT(4); break;
        case 2: AFID_FFTYT(2); break;
        default: AFID_FFTYT(1); break;
      }
#undef AFID_FFTYT
      c->launches++;
      return cudaGetLastError();
    }
  }
  const size_t sm = (size_t)tk * ls + (size_t)g.ny * sizeof(typename cplx<R>::T);
#define AFID_FFTY(TKV)                                                                        \
  do {                                                                                        \
    auto kf = inv ? (gen ? k_fft_y<R, true, TKV, true> : k_fft_y<R, true, TKV, false>)       \
                  : (gen ? k_fft_y<R, false, TKV, true> : k_fft_y<R, false, TKV, false>);    \
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);           \
    kf<<<grd, thr, sm, c->stream>>>(g, spec, tw, skip, nullptr, 0);                                    \
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
  // tangent-form twiddles for the FP64 transform where the context has them
  const bool tan = sizeof(R) == sizeof(double) && c->xtan64[0] != nullptr;
  const int tlen = tan ? c->xtan_len : 0;
  const int tabw = tan ? std::max(g.M, (tlen + 1) / 2) : g.M;
  const size_t sm = (size_t)lines * line_smem<R>(g.M) + (size_t)(g.nx + tabw + g.M / 2 + 1) * sizeof(typename cplx<R>::T);
  const int blocks = ceil_div((long long)g.nz * g.ny, lines);
  const bool gen = !is_pow2(g.M);
  const double* tt = tan ? c->xtan64[0] : nullptr;
  if (rhs) {
    auto kf = gen ? k_r2c_x<R, MODE_RHS, true> : (tan ? k_r2c_x<R, MODE_RHS, false, true> : k_r2c_x<R, MODE_RHS, false>);
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, rhs, u, v, w, scale, spec, tw, c->scal,
                                             want_stats, skip, (int)dev_s, tt, tlen);
  } else {
    auto kf = gen ? k_r2c_x<R, MODE_DIV, true> : (tan ? k_r2c_x<R, MODE_DIV, false, true> : k_r2c_x<R, MODE_DIV, false>);
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, rhs, u, v, w, scale, spec, tw, c->scal,
                                             want_stats, skip, (int)dev_s, tt, tlen);
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
  // tangent-form twiddles for the FP64 transform where the context has them
  const bool tan = sizeof(R) == sizeof(double) && c->xtan64[1] != nullptr;
  const int tlen = tan ? c->xtan_len : 0;
  const int tabw = tan ? std::max(g.M, (tlen + 1) / 2) : g.M;
  const size_t sm = (size_t)lines * line_smem<R>(g.M) + (size_t)(g.nx + tabw + g.M / 2 + 1) * sizeof(typename cplx<R>::T);
  const int blocks = ceil_div((long long)g.nz * g.ny, lines);
  const double scale = 1.0 / ((double)g.nx * (double)g.ny);
  const bool gen = !is_pow2(g.M);
  auto kf = gen ? (mode == 1 ? k_c2r_x<R, 1, true> : (mode == 2 ? k_c2r_x<R, 2, true> : k_c2r_x<R, 0, true>))
                : (mode == 1 ? k_c2r_x<R, 1, false>
                             : (mode == 2 ? k_c2r_x<R, 2, false> : (tan ? k_c2r_x<R, 0, false, true> : k_c2r_x<R, 0, false>)));
  cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, spec, tw, scale, phi, skip, part, c->scal + S_PHIMEAN,
                                           sizeof(R) == sizeof(float) ? c->dprev : nullptr,
                                           tan ? c->xtan64[1] : nullptr, tlen);
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
  if (c->warp_tridiag) {  // long-column variant: one warp per system
    ProfScope ps(c, KF_THOMAS);
    const int nm = g.ny * (g.M + 1), wpb = warps_per_block(g.nz);
    const size_t wsm = (size_t)32 * wpb * 5 * warp_rows(g.nz) * sizeof(double);
    cudaFuncSetAttribute(k_tridiag_warp<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
    k_tridiag_warp<double2><<<ceil_div(nm, wpb), 32 * wpb, wsm, c->stream>>>(
        g, c->m, spec, nullptr, nm, c->lamx, c->lamy, nullptr);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
  } else {
    ProfScope ps(c, KF_THOMAS);
    const int grd = ceil_div((long long)g.ny * (g.M + 1), 128);
    k_thomas<double><<<grd, 128, 0, c->stream>>>(g, c->m, spec, c->mtab64, c->m.pa, c->m.pc,
                                                 c->lamx, c->lamy, 0.0, nullptr);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
  }
  {
    ProfScope ps(c, KF_ZERO);
    int zt;
    size_t zs;
    launch_zero_mode_threads(g, &zt, &zs);
    k_zero_mode<double><<<1, zt, zs, c->stream>>>(g, c->m, spec, c->scal, nullptr);
  }
  c->launches++;
  if ((e = cudaGetLastError())) return e;
  if ((e = run_fft_y<double>(c, spec, c->twy64, true, nullptr))) return e;
  return run_c2r<double>(c, spec, c->twx64, phi, 0, nullptr, nullptr);
}

// FP32 spectral solve of `src` (FP64) for the mixed-precision refinement:
// phi = delta (first) or phi += delta, with per-block partials of ||delta||^2
// and of sum dzc phi in c->part2; every kernel returns at once when *skip != 0.
cudaError_t spectral_solve_fp32(afid_ctx* c, const double* b, const double* phi_in, double* phi,
                                const double* skip, int it, bool stats) {
  const bool first = it == 0;
  const Grid& g = c->g;
  float2* spec = static_cast<float2*>(c->spec);
  cudaError_t e;
  {
    ProfScope ps(c, KF_R2C);
    const int T = g.M / 8, lines = r2c_lines<float>(g);
    // the update stages its stencil rows when every block lies in one plane
    const int mode = it == 0 ? R32_FIRST
                             : (it == 1 ? R32_RESID : (g.ny % lines == 0 && T <= 256 ? R32_RESUPD_ST : R32_RESUPD));
    const size_t sm = (size_t)r2c32_front_words(mode, lines, g.nx, pad8(g.M) + 1) * sizeof(float2) +
                      (size_t)(g.nx + g.M) * sizeof(float2);
    const int blocks = ceil_div((long long)g.nz * g.ny, lines);
    const bool gen = !is_pow2(g.M);
    auto pick = [&](auto k0, auto k1, auto k2, auto k3) {
      return mode == R32_FIRST ? k0 : (mode == R32_RESID ? k1 : (mode == R32_RESUPD ? k2 : k3));
    };
    auto kf = gen ? pick(k_r2c_x32<R32_FIRST, true>, k_r2c_x32<R32_RESID, true>, k_r2c_x32<R32_RESUPD, true>,
                         k_r2c_x32<R32_RESUPD_ST, true>)
                  : pick(k_r2c_x32<R32_FIRST, false>, k_r2c_x32<R32_RESID, false>, k_r2c_x32<R32_RESUPD, false>,
                         k_r2c_x32<R32_RESUPD_ST, false>);
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<blocks, lines * T, sm, c->stream>>>(g, c->m, b, phi_in, spec, c->twx32, c->scal, c->part3,
                                             stats ? 1 : 0, skip, c->rres, c->dprev, c->cff);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
  }
  if (first && (e = bstats_final(c))) return e;
  if (c->fuse_yt) {  // small nz: y transforms and wall-normal solves in one kernel per kx column
    {
      ProfScope ps(c, KF_YT);
      auto kf = is_pow2(g.ny) ? k_yfft_thomas32<false> : k_yfft_thomas32<true>;
      kf<<<g.M + 1, c->yt_threads, c->yt_smem, c->stream>>>(g, c->m, spec, c->twy32, c->mtabt32, c->mtab64,
                                                            c->pa32, c->pc32, c->lowslot, c->yt_lmax,
                                                            c->scal, skip);
      c->launches++;
      if ((e = cudaGetLastError())) return e;
    }
    return run_c2r<float>(c, spec, c->twx32, phi, first ? 2 : 1, skip, c->part2);
  }
  if ((e = run_fft_y<float>(c, spec, c->twy32, false, skip))) return e;
  {
    ProfScope ps(c, KF_THOMAS);
    const int grd = ceil_div((long long)g.ny * (g.M + 1), 128);
    k_thomas_mixed<<<grd, 128, 0, c->stream>>>(g, c->m, spec, c->mtab32, c->mtab64, c->pa32,
                                               c->pc32, c->lowslot, c->nlow, c->low_scratch, skip);
    c->launches++;
    if ((e = cudaGetLastError())) return e;
    if (c->nlow > 0) {
      const int wpb = warps_per_block(g.nz);
      const size_t wsm = (size_t)32 * wpb * 5 * warp_rows(g.nz) * sizeof(double);
      cudaFuncSetAttribute(k_tridiag_warp<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
      k_tridiag_warp<float2><<<ceil_div(c->nlow, wpb), 32 * wpb, wsm, c->stream>>>(
          g, c->m, spec, c->low_modes, c->nlow, c->lamx, c->lamy, skip);
      c->launches++;
      if ((e = cudaGetLastError())) return e;
    }
  }
  {
    ProfScope ps(c, KF_ZERO);
    int zt;
    size_t zs;
    launch_zero_mode_threads(g, &zt, &zs);
    k_zero_mode<float><<<1, zt, zs, c->stream>>>(g, c->m, spec, c->scal, skip);
  }
  c->launches++;
  if ((e = cudaGetLastError())) return e;
  if ((e = run_fft_y<float>(c, spec, c->twy32, true, skip))) return e;
  return run_c2r<float>(c, spec, c->twx32, phi, first ? 2 : 1, skip, c->part2);
}

// Tables of fft_line_tan_ix for a power-of-two N >= 64 (host, FP64), in pass
// order: per radix-8 pass of span p > 1, 16 rows of p doubles (layout in
// stockham_pass8_tan), then for a last radix-4 pass 7 rows of p doubles
// (stockham_pass4_tan), or for a last radix-2 pass its p complex twiddles
// w = tw[k N/(2p)] as pass_twiddles lays them out (the inverse pass conjugates
// them itself). tw: exp(-2 pi i m/N), m < N. The
// inverse tables take W = conj(w). Returns the length in doubles; out may be
// null to size it.
int tan_tables(int N, const double2* tw, bool inv, double* out) {
  const double h = 0.70710678118654752440;  // the 1/sqrt2 of the radix-8 butterfly
  int off = 0, p = 1, n2 = N;
  while (n2 >= 8) {
    if (p > 1) {
      const int step = N / (8 * p);
      for (int k = 0; out && k < p; ++k) {
        double kap[8] = {1.0}, tt[8] = {0.0};
        unsigned long long fl = 0;
        for (int r = 1; r < 8; ++r) {
          const double2 w = tw[r * k * step];
          const double cs = w.x, sn = inv ? -w.y : w.y;
          if (std::fabs(cs) >= std::fabs(sn)) {
            kap[r] = cs;
            tt[r] = sn / cs;
          } else {  // W = i sin (1 - i cot): the input is rotated by i
            kap[r] = sn;
            tt[r] = -cs / sn;
            fl |= 1ull << r;
          }
        }
        for (int r = 1; r < 8; ++r) out[off + (r - 1) * p + k] = tt[r];
        out[off + 7 * p + k] = kap[4];
        out[off + 8 * p + k] = kap[6] / kap[2];
        out[off + 9 * p + k] = kap[2];
        out[off + 10 * p + k] = kap[5] / kap[1];
        out[off + 11 * p + k] = kap[7] / kap[3];
        out[off + 12 * p + k] = kap[3] / kap[1];
        out[off + 13 * p + k] = kap[1];
        out[off + 14 * p + k] = h * kap[1];
        double flb;
        std::memcpy(&flb, &fl, sizeof(flb));
        out[off + 15 * p + k] = flb;
      }
      off += 16 * p;
    }
    p *= 8;
    n2 /= 8;
  }
  if (n2 == 4) {  // last radix-4 pass in tangent form: 7 rows of p (stockham_pass4_tan)
    const int step = N / (4 * p);
    for (int k = 0; out && k < p; ++k) {
      double kap[4] = {1.0}, tt[4] = {0.0};
      unsigned long long fl = 0;
      for (int r = 1; r < 4; ++r) {
        const double2 w = tw[r * k * step];
        const double cs = w.x, sn = inv ? -w.y : w.y;
        if (std::fabs(cs) >= std::fabs(sn)) {
          kap[r] = cs;
          tt[r] = sn / cs;
        } else {
          kap[r] = sn;
          tt[r] = -cs / sn;
          fl |= 1ull << r;
        }
      }
      for (int r = 1; r < 4; ++r) out[off + (r - 1) * p + k] = tt[r];
      out[off + 3 * p + k] = kap[2];
      out[off + 4 * p + k] = kap[3] / kap[1];
      out[off + 5 * p + k] = kap[1];
      double flb;
      std::memcpy(&flb, &fl, sizeof(flb));
      out[off + 6 * p + k] = flb;
    }
    off += 7 * p;
  } else if (n2 == 2) {
    const int R = n2, step = N / (p * R);
    for (int r = 1; out && r < R; ++r)
      for (int k = 0; k < p; ++k) {
        const double2 w = tw[r * k * step];
        out[off + 2 * ((r - 1) * p + k)] = w.x;
        out[off + 2 * ((r - 1) * p + k) + 1] = w.y;
      }
    off += 2 * (R - 1) * p;
  }
  return off;
}

int c2r_blocks(const Grid& g) {
  const int T = g.M / 8;
  int lines = 256 / T;
  if (lines < 1) lines = 1;
  return ceil_div((long long)g.nz * g.ny, lines);
}
}  // namespace afid
