// Shared-memory Stockham FFT building blocks (radix 8 / 4 / 2 / 3 / 5) for sm_103a.
//
// One line of N = 2^a 3^b 5^c complex points (8 | N) lives in shared memory with one padding
// slot every 8 elements (pad(m) = m + m/8), so that the stride-R writes of a
// Stockham pass spread over the banks. Each thread owns 8 complex values per
// pass: one radix-8 butterfly, two radix-4 or four radix-2 butterflies (up to
// three radix-3 or two radix-5 butterflies). A line is transformed by N/8
// threads; the pass sequence is radix 8 while at least three factors of two
// remain, then one radix-4 or radix-2 pass, then the factors 3 and 5 (the
// first pass needs no twiddles, so the large radix goes first).
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / NT) of the table length
// NT (a multiple of N), computed on the host in FP64; the transform of length
// N reads it with index stride NT / N. Forward = exp(-), inverse = exp(+)
// (conjugated twiddles), both unnormalised.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace afid {

template <typename R> struct cplx;
template <> struct cplx<double> { using T = double2; };
template <> struct cplx<float> { using T = float2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return C{a.x * s, a.y * s}; }

__host__ __device__ __forceinline__ int pad8(int m) { return m + (m >> 3); }

// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot_mi(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
  C t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = rot_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* a) {
  using R = decltype(a[0].x);
  const R h = (R)0.70710678118654752440;  // 1/sqrt(2)
  // even / odd halves
  dft4<INV>(a[0], a[2], a[4], a[6]);
  dft4<INV>(a[1], a[3], a[5], a[7]);
  // twiddle the odd half by w8^k, k = 1, 2, 3; the 1/sqrt(2) of w8 and w8^3
  // is applied inside the final additions (one FMA each instead of a
  // multiplication and an addition)
  C o1 = a[3], o2 = a[5], o3 = a[7];
  if (!INV) {
    o1 = C{o1.x + o1.y, o1.y - o1.x};
    o3 = C{o3.y - o3.x, -(o3.x + o3.y)};
  } else {
    o1 = C{o1.x - o1.y, o1.x + o1.y};
    o3 = C{-(o3.x + o3.y), o3.x - o3.y};
  }
  o2 = rot_mi<INV>(o2);
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1];
  a[0] = cadd(e0, o0);
  a[4] = csub(e0, o0);
  a[1] = C{fma(o1.x, h, e1.x), fma(o1.y, h, e1.y)};
  a[5] = C{fma(-o1.x, h, e1.x), fma(-o1.y, h, e1.y)};
  a[2] = cadd(e2, o2);
  a[6] = csub(e2, o2);
  a[3] = C{fma(o3.x, h, e3.x), fma(o3.y, h, e3.y)};
  a[7] = C{fma(-o3.x, h, e3.x), fma(-o3.y, h, e3.y)};
}

// 3-point DFT: y0 = a0 + s, y1,2 = a0 - s/2 -/+ i (sqrt(3)/2) d (forward),
// s = a1 + a2, d = a1 - a2; the inverse flips the sign of i.
template <bool INV, typename C> __device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
  using R = decltype(a0.x);
  const R c = (R)0.86602540378443864676;  // sqrt(3)/2
  const C s = cadd(a1, a2), d = csub(a1, a2);
  const C t = C{fma((R)-0.5, s.x, a0.x), fma((R)-0.5, s.y, a0.y)};
  a0 = cadd(a0, s);
  const C u = C{c * d.x, c * d.y};  // (sqrt(3)/2) d
  // -i u = (u.y, -u.x), +i u = (-u.y, u.x)
  if (!INV) {
    a1 = C{t.x + u.y, t.y - u.x};
    a2 = C{t.x - u.y, t.y + u.x};
  } else {
    a1 = C{t.x - u.y, t.y + u.x};
    a2 = C{t.x + u.y, t.y - u.x};
  }
}

// 5-point DFT with w = exp(-2 pi i/5): s1 = a1 + a4, d1 = a1 - a4, s2 = a2 + a3,
// d2 = a2 - a3; t1 = a0 + c1 s1 + c2 s2, t2 = a0 + c2 s1 + c1 s2,
// u1 = n1 d1 + n2 d2, u2 = n2 d1 - n1 d2 (c_m = cos(2 pi m/5), n_m = sin(2 pi m/5));
// y1 = t1 - i u1, y4 = t1 + i u1, y2 = t2 - i u2, y3 = t2 + i u2 (forward; the
// inverse flips the sign of i).
template <bool INV, typename C> __device__ __forceinline__ void dft5(C* a) {
  using R = decltype(a[0].x);
  const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
  const R n1 = (R)0.95105651629515357212, n2 = (R)0.58778525229247312917;
  const C s1 = cadd(a[1], a[4]), d1 = csub(a[1], a[4]);
  const C s2 = cadd(a[2], a[3]), d2 = csub(a[2], a[3]);
  const C t1 = C{fma(c2, s2.x, fma(c1, s1.x, a[0].x)), fma(c2, s2.y, fma(c1, s1.y, a[0].y))};
  const C t2 = C{fma(c1, s2.x, fma(c2, s1.x, a[0].x)), fma(c1, s2.y, fma(c2, s1.y, a[0].y))};
  const C u1 = C{fma(n2, d2.x, n1 * d1.x), fma(n2, d2.y, n1 * d1.y)};
  const C u2 = C{fma(-n1, d2.x, n2 * d1.x), fma(-n1, d2.y, n2 * d1.y)};
  a[0] = cadd(a[0], cadd(s1, s2));
  const R sg = INV ? (R)-1 : (R)1;  // -i (forward) or +i (inverse) times u
  a[1] = C{fma(sg, u1.y, t1.x), fma(-sg, u1.x, t1.y)};
  a[4] = C{fma(-sg, u1.y, t1.x), fma(sg, u1.x, t1.y)};
  a[2] = C{fma(sg, u2.y, t2.x), fma(-sg, u2.x, t2.y)};
  a[3] = C{fma(-sg, u2.y, t2.x), fma(sg, u2.x, t2.y)};
}

// Shared-memory slot of point m of a line: padded line (one slot every 8
// points), or column c of a tile of TK interleaved lines (point m of every
// line in one row of TK slots, as a TMA box lands in shared memory).
struct PadIx {
  __device__ __forceinline__ int operator()(int m) const { return pad8(m); }
};
template <int TK> struct ColIx {
  int c;
  __device__ __forceinline__ int operator()(int m) const { return m * TK + c; }
};

// One Stockham pass of radix R (8, 4, 2, 3 or 5) on a shared-memory line `buf`
// of N points (slot of point m: ix(m)), span p (product of the radices of the
// passes already done). `t` in [0, N/8) is the thread's index within the
// line (8 | N); it takes butterflies j = t + b N/8 < N/R, b < ceil(8/R). All
// reads happen before the barrier, all writes after it, so the pass is in
// place. The caller guarantees that every thread of the block calls this
// (barriers inside). PT: `tw` is this pass's own table, entry (r - 1) p + k =
// w^(r k N/(p R)) (see pass_twiddles), so that lanes with consecutive k read
// consecutive entries. XM (R = 8, first pass only): butterfly j writes its
// outputs in the order r ^ (j & XM) instead of r, the same values to the same
// slots: in a tile of TK-wide rows (ColIx<TK>) the lanes of a warp hold 32 / TK
// consecutive j, whose outputs 8 j + r lie 8 rows apart, all in the same banks
// when the rows are 32 or 64 bytes wide; rotating r spreads each store over
// the 128 bytes of banks (XM = 3 for TK = 4, 1 for TK = 8).
template <int R, bool INV, typename C, typename IX, bool PT = false, int XM = 0>
__device__ __forceinline__ void stockham_pass_ix(C* buf, int N, int p, const C* tw, int twstride,
                                                 int t, bool active, IX ix) {
  constexpr int B = (8 + R - 1) / R;  // butterflies per thread (at most)
  C x[B * R];
  const int nb = N / R, T = N / 8;
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * T;
      if ((8 % R == 0) || j < nb) {
#pragma unroll
        for (int r = 0; r < R; ++r) x[b * R + r] = buf[ix(j + r * nb)];
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * T;
      if ((8 % R == 0) || j < nb) {
        // the radix-8/4/2 passes come first, so p is a power of two there
        const int k = (8 % R == 0) ? (j & (p - 1)) : j % p;
        C* y = x + b * R;
        if (p > 1) {
          const int step = (N / (p * R)) * twstride;
#pragma unroll
          for (int r = 1; r < R; ++r) {
            const C w = PT ? tw[(r - 1) * p + k] : tw[r * k * step];
            y[r] = INV ? cmulc(y[r], w) : cmul(y[r], w);
          }
        }
        if (R == 8) dft8<INV>(y);
        if (R == 4) dft4<INV>(y[0], y[1], y[2], y[3]);
        if (R == 2) dft2<INV>(y[0], y[1]);
        if (R == 3) dft3<INV>(y[0], y[1], y[2]);
        if (R == 5) dft5<INV>(y);
        const int o = (j - k) * R + k;
        if constexpr (XM != 0 && R == 8) {
          const int sx = j & XM;  // y[r] <- y[r ^ sx], then slot r ^ sx gets y[r]
          auto swp = [](C& a, C& b2) {
            const C tmp = a;
            a = b2;
            b2 = tmp;
          };
          if (sx & 1) {
#pragma unroll
            for (int r = 0; r < 8; r += 2) swp(y[r], y[r + 1]);
          }
          if ((XM & 2) && (sx & 2)) {
            swp(y[0], y[2]);
            swp(y[1], y[3]);
            swp(y[4], y[6]);
            swp(y[5], y[7]);
          }
#pragma unroll
          for (int r = 0; r < 8; ++r) buf[ix(o + (r ^ sx) * p)] = y[r];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) buf[ix(o + r * p)] = y[r];
        }
      }
    }
  }
  __syncthreads();
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void stockham_pass(C* buf, int N, int p, const C* tw, int twstride,
                                              int t, bool active) {
  stockham_pass_ix<R, INV>(buf, N, p, tw, twstride, t, active, PadIx{});
}

// Full N-point transform of one line; N = 2^a 3^b 5^c with 8 | N. The
// radix-8 passes go first (the first pass needs no twiddles), then one radix-4
// or radix-2 pass for the rest of the power of two, then the radix-3 and
// radix-5 passes.
// GEN = false compiles the power-of-two passes only (N = 2^a): no radix-3/5
// code, and so no registers held for it.
template <bool INV, bool GEN, typename C, typename IX>
__device__ __forceinline__ void fft_line_ix(C* buf, int N, const C* tw, int twstride, int t,
                                            bool active, IX ix) {
  int p = 1;
  int n2 = N & -N;  // power-of-two part of N
  int rest = N / n2;
  while (n2 >= 8) {
    stockham_pass_ix<8, INV>(buf, N, p, tw, twstride, t, active, ix);
    p *= 8;
    n2 /= 8;
  }
  if (n2 == 4) {
    stockham_pass_ix<4, INV>(buf, N, p, tw, twstride, t, active, ix);
    p *= 4;
  } else if (n2 == 2) {
    stockham_pass_ix<2, INV>(buf, N, p, tw, twstride, t, active, ix);
    p *= 2;
  }
  if constexpr (GEN) {
    while (rest % 3 == 0) {
      stockham_pass_ix<3, INV>(buf, N, p, tw, twstride, t, active, ix);
      p *= 3;
      rest /= 3;
    }
    while (rest % 5 == 0) {
      stockham_pass_ix<5, INV>(buf, N, p, tw, twstride, t, active, ix);
      p *= 5;
      rest /= 5;
    }
  }
}

// Per-pass twiddle tables of a power-of-two transform of length N (8 | N), in
// pass order, for the passes with span p > 1: R - 1 rows of p entries each,
// entry (r - 1) p + k = tw[r k N/(p R) twstride] (tw read with the stride of
// its length over N). The rows add up to N - 8 entries (each pass's (R - 1) p
// is the next span minus this one). Filled by the threads of the block (tid
// of nthr); the caller synchronises before use.
template <typename C>
__device__ __forceinline__ void pass_twiddles(C* out, const C* __restrict__ tw, int N, int twstride, int tid,
                                              int nthr) {
  int off = 0, p = 1, n2 = N;
  while (n2 > 1) {
    const int R = n2 >= 8 ? 8 : n2;
    if (p > 1) {
      const int step = N / (p * R), n = (R - 1) * p;
      for (int i = tid; i < n; i += nthr) {
        const int r = i / p + 1, k = i - (r - 1) * p;
        out[off + i] = tw[r * k * step * twstride];
      }
      off += n;
    }
    p *= R;
    n2 /= R;
  }
}

// fft_line_ix for a power-of-two N with the per-pass twiddle tables of
// pass_twiddles in `tabs`: the same arithmetic, the same results.
// XM: see stockham_pass_ix (the first pass).
template <bool INV, int XM, typename C, typename IX>
__device__ __forceinline__ void fft_line_pt_ix(C* buf, int N, const C* tabs, int t, bool active, IX ix) {
  stockham_pass_ix<8, INV, C, IX, true, XM>(buf, N, 1, tabs, 1, t, active, ix);
  int p = 8, n2 = N / 8, off = 0;
  while (n2 >= 8) {
    stockham_pass_ix<8, INV, C, IX, true>(buf, N, p, tabs + off, 1, t, active, ix);
    if (p > 1) off += 7 * p;
    p *= 8;
    n2 /= 8;
  }
  if (n2 == 4) stockham_pass_ix<4, INV, C, IX, true>(buf, N, p, tabs + off, 1, t, active, ix);
  else if (n2 == 2) stockham_pass_ix<2, INV, C, IX, true>(buf, N, p, tabs + off, 1, t, active, ix);
}

// FP64 radix-8 pass of span p > 1 with its twiddles in tangent form. The
// twiddle W_r = exp(+-2 pi i r k / (8p)) of input r is written kappa_r (1 + i t_r)
// with |t_r| <= 1: kappa_r = cos, t_r = tan where |cos| >= |sin|; elsewhere the
// input is first rotated by i (exact: a swap and a sign) and W_r / i =
// sin (1 - i cot), kappa_r = sin, t_r = -cot. The product costs two FMAs instead
// of four; the seven factors kappa_r go into the butterfly's own additions,
// which become FMAs (kappa_4 and kappa_2 into the even 4-point DFT, ratios
// kappa_6/kappa_2, kappa_5/kappa_1, kappa_7/kappa_3, kappa_3/kappa_1 inside
// it, kappa_1 and kappa_1/sqrt2 into the final combination): 66 FP64
// operations per butterfly of 8 points instead of 80, the same DFT (the
// arithmetic order differs, the results agree to rounding). `tab` is this
// pass's table, 16 rows of p doubles ([row][k]): rows 0..6 t_1..t_7, 7 kappa_4,
// 8 kappa_6/kappa_2, 9 kappa_2, 10 kappa_5/kappa_1, 11 kappa_7/kappa_3,
// 12 kappa_3/kappa_1, 13 kappa_1, 14 kappa_1/sqrt2, 15 the rotated inputs as
// a bit mask (bit r) in the bits of a double. Forward and inverse passes take
// their own tables. Built by tan_tables (host).
template <bool INV, typename IX>
__device__ __forceinline__ void stockham_pass8_tan(double2* buf, int N, int p, const double* tab, int t,
                                                   bool active, IX ix) {
  double2 x[8];
  const int nb = N / 8;
  if (active) {
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = buf[ix(t + r * nb)];
  }
  __syncthreads();
  if (active) {
    const int k = t & (p - 1);
    const unsigned long long fl = (unsigned long long)__double_as_longlong(tab[15 * p + k]);
    // z_r: input r times (1 + i t_r), after the rotation by i where flagged
    auto tw = [&](int r) {
      const double tr = tab[(r - 1) * p + k];
      const bool rot = (fl >> r) & 1ull;
      // (a, b) = i x where rotated (integer sign flip and selects), else x
      const double nyv = __longlong_as_double(__double_as_longlong(x[r].y) ^ (long long)0x8000000000000000ull);
      const double a = rot ? nyv : x[r].x;
      const double b = rot ? x[r].x : x[r].y;
      return double2{fma(-tr, b, a), fma(tr, a, b)};
    };
    // even 4-point DFT of (x0, kappa_2 z2, kappa_4 z4, kappa_6 z6), formed
    // before the odd inputs are touched (fewer live registers)
    double2 e0, e1, e2, e3;
    {
      const double2 z2 = tw(2), z4 = tw(4), z6 = tw(6);
      const double k4 = tab[7 * p + k], r26 = tab[8 * p + k], k2 = tab[9 * p + k];
      const double2 t0{fma(k4, z4.x, x[0].x), fma(k4, z4.y, x[0].y)};
      const double2 t1{fma(-k4, z4.x, x[0].x), fma(-k4, z4.y, x[0].y)};
      const double2 t2{fma(r26, z6.x, z2.x), fma(r26, z6.y, z2.y)};
      const double2 t3 = rot_mi<INV>(double2{fma(-r26, z6.x, z2.x), fma(-r26, z6.y, z2.y)});
      e0 = double2{fma(k2, t2.x, t0.x), fma(k2, t2.y, t0.y)};
      e2 = double2{fma(-k2, t2.x, t0.x), fma(-k2, t2.y, t0.y)};
      e1 = double2{fma(k2, t3.x, t1.x), fma(k2, t3.y, t1.y)};
      e3 = double2{fma(-k2, t3.x, t1.x), fma(-k2, t3.y, t1.y)};
    }
    // odd 4-point DFT of (kappa_1 z1, kappa_3 z3, kappa_5 z5, kappa_7 z7), kappa_1 factored out
    double2 o0, o1, o2, o3;
    {
      const double2 z1 = tw(1), z3 = tw(3), z5 = tw(5), z7 = tw(7);
      const double r15 = tab[10 * p + k], r37 = tab[11 * p + k], r13 = tab[12 * p + k];
      const double2 u0{fma(r15, z5.x, z1.x), fma(r15, z5.y, z1.y)};
      const double2 u1{fma(-r15, z5.x, z1.x), fma(-r15, z5.y, z1.y)};
      const double2 u2{fma(r37, z7.x, z3.x), fma(r37, z7.y, z3.y)};
      const double2 u3 = rot_mi<INV>(double2{fma(-r37, z7.x, z3.x), fma(-r37, z7.y, z3.y)});
      o0 = double2{fma(r13, u2.x, u0.x), fma(r13, u2.y, u0.y)};
      o2 = double2{fma(-r13, u2.x, u0.x), fma(-r13, u2.y, u0.y)};
      o1 = double2{fma(r13, u3.x, u1.x), fma(r13, u3.y, u1.y)};
      o3 = double2{fma(-r13, u3.x, u1.x), fma(-r13, u3.y, u1.y)};
    }
    // w8 twiddles of the odd outputs (the 1/sqrt2 is in hk1), as in dft8
    if (!INV) {
      o1 = double2{o1.x + o1.y, o1.y - o1.x};
      o3 = double2{o3.y - o3.x, -(o3.x + o3.y)};
    } else {
      o1 = double2{o1.x - o1.y, o1.x + o1.y};
      o3 = double2{-(o3.x + o3.y), o3.x - o3.y};
    }
    const double2 q2 = rot_mi<INV>(o2);
    const double k1 = tab[13 * p + k], hk1 = tab[14 * p + k];
    double2 y[8];
    y[0] = double2{fma(k1, o0.x, e0.x), fma(k1, o0.y, e0.y)};
    y[4] = double2{fma(-k1, o0.x, e0.x), fma(-k1, o0.y, e0.y)};
    y[1] = double2{fma(hk1, o1.x, e1.x), fma(hk1, o1.y, e1.y)};
    y[5] = double2{fma(-hk1, o1.x, e1.x), fma(-hk1, o1.y, e1.y)};
    y[2] = double2{fma(k1, q2.x, e2.x), fma(k1, q2.y, e2.y)};
    y[6] = double2{fma(-k1, q2.x, e2.x), fma(-k1, q2.y, e2.y)};
    y[3] = double2{fma(hk1, o3.x, e3.x), fma(hk1, o3.y, e3.y)};
    y[7] = double2{fma(-hk1, o3.x, e3.x), fma(-hk1, o3.y, e3.y)};
    const int o = (t - k) * 8 + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[ix(o + r * p)] = y[r];
  }
  __syncthreads();
}

// The last radix-4 pass (span p = N/4) in tangent form: two 4-point
// butterflies per thread, twiddles kappa_r (1 + i t_r) as in stockham_pass8_tan;
// kappa_2 and kappa_1 go into the butterfly's FMAs, kappa_3 as kappa_3/kappa_1:
// 22 FP64 operations per butterfly instead of 28. `tab`: 7 rows of p doubles,
// t_1..t_3, kappa_2, kappa_3/kappa_1, kappa_1, the rotation mask (bits 1..3).
template <bool INV, typename IX>
__device__ __forceinline__ void stockham_pass4_tan(double2* buf, int N, int p, const double* tab, int t,
                                                   bool active, IX ix) {
  double2 x[8];
  const int nb = N / 4, T = N / 8;
  if (active) {
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int r = 0; r < 4; ++r) x[b * 4 + r] = buf[ix(t + b * T + r * nb)];
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = t + b * T;
      const int k = j & (p - 1);
      const unsigned long long fl = (unsigned long long)__double_as_longlong(tab[6 * p + k]);
      const double2* xb = x + b * 4;
      auto tw = [&](int r) {
        const double tr = tab[(r - 1) * p + k];
        const bool rot = (fl >> r) & 1ull;
        const double nyv = __longlong_as_double(__double_as_longlong(xb[r].y) ^ (long long)0x8000000000000000ull);
        const double a = rot ? nyv : xb[r].x;
        const double bb = rot ? xb[r].x : xb[r].y;
        return double2{fma(-tr, bb, a), fma(tr, a, bb)};
      };
      const double2 z1 = tw(1), z2 = tw(2), z3 = tw(3);
      const double k2 = tab[3 * p + k], r13 = tab[4 * p + k], k1 = tab[5 * p + k];
      const double2 t0{fma(k2, z2.x, xb[0].x), fma(k2, z2.y, xb[0].y)};
      const double2 t1{fma(-k2, z2.x, xb[0].x), fma(-k2, z2.y, xb[0].y)};
      const double2 t2{fma(r13, z3.x, z1.x), fma(r13, z3.y, z1.y)};
      const double2 t3 = rot_mi<INV>(double2{fma(-r13, z3.x, z1.x), fma(-r13, z3.y, z1.y)});
      const int o = (j - k) * 4 + k;
      buf[ix(o)] = double2{fma(k1, t2.x, t0.x), fma(k1, t2.y, t0.y)};
      buf[ix(o + 2 * p)] = double2{fma(-k1, t2.x, t0.x), fma(-k1, t2.y, t0.y)};
      buf[ix(o + p)] = double2{fma(k1, t3.x, t1.x), fma(k1, t3.y, t1.y)};
      buf[ix(o + 3 * p)] = double2{fma(-k1, t3.x, t1.x), fma(-k1, t3.y, t1.y)};
    }
  }
  __syncthreads();
}

// Transform of a power-of-two line of N >= 64 FP64 points with the radix-8
// passes of span p > 1 in tangent form: the first pass (no twiddles) as in
// fft_line, then stockham_pass8_tan per radix-8 pass, then a last radix-4 pass
// in tangent form (stockham_pass4_tan) or a radix-2 pass with its per-pass
// table of pass_twiddles (complex). Layout: tan_tables (host).
template <bool INV, typename IX>
__device__ __forceinline__ void fft_line_tan_ix(double2* buf, int N, const double* tab, int t, bool active,
                                                IX ix) {
  stockham_pass_ix<8, INV>(buf, N, 1, reinterpret_cast<const double2*>(tab), 1, t, active, ix);
  int p = 8, n2 = N / 8, off = 0;
  while (n2 >= 8) {
    stockham_pass8_tan<INV>(buf, N, p, tab + off, t, active, ix);
    off += 16 * p;
    p *= 8;
    n2 /= 8;
  }
  if (n2 == 4) stockham_pass4_tan<INV>(buf, N, p, tab + off, t, active, ix);
  else if (n2 == 2)
    stockham_pass_ix<2, INV, double2, IX, true>(buf, N, p, reinterpret_cast<const double2*>(tab + off), 1, t,
                                                active, ix);
}

template <bool INV, typename C>
__device__ __forceinline__ void fft_line_pt(C* buf, int N, const C* tabs, int t, bool active) {
  fft_line_pt_ix<INV, 0>(buf, N, tabs, t, active, PadIx{});
}

template <bool INV, bool GEN, typename C>
__device__ __forceinline__ void fft_line(C* buf, int N, const C* tw, int twstride, int t, bool active) {
  fft_line_ix<INV, GEN>(buf, N, tw, twstride, t, active, PadIx{});
}

// The same transform when the thread already holds, in x[0..7], the points
// t + r N/8 of its line (the inputs of its butterfly in the first radix-8
// pass, which takes no twiddles): that pass runs from registers and writes
// its outputs to the padded line, saving one shared-memory round trip; the
// remaining passes follow as in fft_line. The arithmetic is that of
// fft_line, in the same order. Every thread of the block calls it (barriers).
// PT (power-of-two N only): `tw` holds the per-pass tables of pass_twiddles.
template <bool INV, bool GEN, bool PT = false, typename C>
__device__ __forceinline__ void fft_line_from_regs(C* buf, int N, C* x, const C* tw, int twstride, int t,
                                                   bool active) {
  static_assert(!(PT && GEN), "per-pass tables cover power-of-two lengths");
  if (active) {
    dft8<INV>(x);
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[pad8(8 * t + r)] = x[r];
  }
  __syncthreads();
  int p = 8;
  int n2 = (N & -N) / 8;
  int rest = N / (N & -N);
  int off = 0;  // PT: offset of the pass's table
  while (n2 >= 8) {
    stockham_pass_ix<8, INV, C, PadIx, PT>(buf, N, p, tw + off, twstride, t, active, PadIx{});
    if (PT) off += 7 * p;
    p *= 8;
    n2 /= 8;
  }
  if (n2 == 4) {
    stockham_pass_ix<4, INV, C, PadIx, PT>(buf, N, p, tw + off, twstride, t, active, PadIx{});
    p *= 4;
  } else if (n2 == 2) {
    stockham_pass_ix<2, INV, C, PadIx, PT>(buf, N, p, tw + off, twstride, t, active, PadIx{});
    p *= 2;
  }
  if constexpr (GEN) {
    while (rest % 3 == 0) {
      stockham_pass<3, INV>(buf, N, p, tw, twstride, t, active);
      p *= 3;
      rest /= 3;
    }
    while (rest % 5 == 0) {
      stockham_pass<5, INV>(buf, N, p, tw, twstride, t, active);
      p *= 5;
      rest /= 5;
    }
  }
}

// The same transform for N a power of two, with the last pass kept in
// registers: after it, out[q] holds point t + q N/8 of the line (q = 0..7),
// the points the caller writes out, so the last shared-memory round trip is
// saved. In the last pass (span p = N/R) butterfly j = t + b N/8 has k = j
// and writes point j + r p, i.e. q = b + r 8/R. The line in shared memory is
// left as the previous pass wrote it. The arithmetic is that of fft_line, in
// the same order. Every thread of the block calls it (barriers).
// PT: `tw` holds the per-pass tables of pass_twiddles.
template <bool INV, bool PT = false, typename C>
__device__ __forceinline__ void fft_line_pow2_to_regs(C* buf, int N, C* out, const C* tw, int twstride,
                                                      int t, bool active) {
  int passes8 = 0, n2 = N;
  while (n2 >= 8) {
    ++passes8;
    n2 /= 8;
  }
  const int last = n2 == 4 ? 4 : (n2 == 2 ? 2 : 8);  // radix of the last pass
  if (last == 8) --passes8;
  int p = 1, off = 0;
  for (int i = 0; i < passes8; ++i) {
    stockham_pass_ix<8, INV, C, PadIx, PT>(buf, N, p, tw + off, twstride, t, active, PadIx{});
    if (PT && p > 1) off += 7 * p;
    p *= 8;
  }
  if (!active) return;
  const int T = N / 8;
  auto run_last = [&](auto radix_tag) {
    constexpr int R = decltype(radix_tag)::value;
    constexpr int B = 8 / R;
    const int nb = N / R;
    C x[8];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * T;
#pragma unroll
      for (int r = 0; r < R; ++r) x[b * R + r] = buf[pad8(j + r * nb)];
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int k = t + b * T;  // j & (p - 1) = j in the last pass
      C* y = x + b * R;
      if (p > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C w = PT ? tw[off + (r - 1) * p + k] : tw[r * k * twstride];
          y[r] = INV ? cmulc(y[r], w) : cmul(y[r], w);
        }
      }
      if (R == 8) dft8<INV>(y);
      if (R == 4) dft4<INV>(y[0], y[1], y[2], y[3]);
      if (R == 2) dft2<INV>(y[0], y[1]);
#pragma unroll
      for (int r = 0; r < R; ++r) out[b + r * B] = y[r];
    }
  };
  if (last == 8) run_last(std::integral_constant<int, 8>{});
  else if (last == 4) run_last(std::integral_constant<int, 4>{});
  else run_last(std::integral_constant<int, 2>{});
}

}  // namespace afid
