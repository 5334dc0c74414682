// C ABI of libafid (declared in include/afid.h): context creation, argument
// validation and the stream-ordered orchestration of the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "afid_internal.cuh"

using namespace afid;

namespace afid {

void metric_fill(int nz, double rdx2, double rdy2, const double* zf, double* out) {
  const int L = nz + 1;
  for (int i = 0; i < METRIC_ARRAYS * L; ++i) out[i] = 0.0;
  double *dzc = out, *rdzc = out + L, *dzf = out + 2 * L, *rdzf = out + 3 * L, *pa = out + 4 * L,
         *pc = out + 5 * L, *ca = out + 6 * L, *cc = out + 7 * L, *fa = out + 8 * L, *fc = out + 9 * L,
         *wlo = out + 10 * L, *whi = out + 11 * L, *pdiag = out + 12 * L;
  for (int k = 0; k < nz; ++k) {
    dzc[k] = zf[k + 1] - zf[k];
    rdzc[k] = 1.0 / dzc[k];
  }
  dzf[0] = 0.5 * dzc[0];
  dzf[nz] = 0.5 * dzc[nz - 1];
  for (int k = 1; k < nz; ++k) dzf[k] = 0.5 * (zf[k] + zf[k + 1]) - 0.5 * (zf[k - 1] + zf[k]);
  for (int k = 0; k <= nz; ++k) rdzf[k] = 1.0 / dzf[k];
  for (int k = 0; k < nz; ++k) {
    if (k > 0) pa[k] = 1.0 / (dzc[k] * dzf[k]);
    if (k < nz - 1) pc[k] = 1.0 / (dzc[k] * dzf[k + 1]);
    ca[k] = 1.0 / (dzc[k] * dzf[k]);
    cc[k] = 1.0 / (dzc[k] * dzf[k + 1]);
  }
  for (int k = 0; k < nz; ++k) pdiag[k] = pa[k] + pc[k] + 2.0 * rdx2 + 2.0 * rdy2;
  for (int k = 1; k < nz; ++k) {
    fa[k] = 1.0 / (dzf[k] * dzc[k - 1]);
    fc[k] = 1.0 / (dzf[k] * dzc[k]);
    wlo[k] = dzc[k - 1] / (2.0 * dzf[k]);
    whi[k] = dzc[k] / (2.0 * dzf[k]);
  }
}

void metric_host(int nz, double rdx2, double rdy2, const double* zf, std::vector<double>& flat,
                 std::vector<size_t>& offs) {
  flat.assign((size_t)METRIC_ARRAYS * (nz + 1), 0.0);
  metric_fill(nz, rdx2, rdy2, zf, flat.data());
  offs.clear();
  for (int a = 0; a < METRIC_ARRAYS; ++a) offs.push_back((size_t)a * (nz + 1));
}

// exp(-2 pi i m / N) with exact octant symmetry
void twiddle(long long m, long long N, double& c, double& s) {
  m %= N;
  const long long q4 = N / 4, q8 = N / 8;
  const long long quad = m / q4, r = m % q4;
  double c0, s0;
  if (r <= q8) {
    const double a = 2.0 * M_PI * (double)r / (double)N;
    c0 = std::cos(a);
    s0 = std::sin(a);
  } else {
    const double a = 2.0 * M_PI * (double)(q4 - r) / (double)N;
    c0 = std::sin(a);
    s0 = std::cos(a);
  }
  if (r == 0) { c0 = 1.0; s0 = 0.0; }
  double cc, ss;
  switch (quad) {
    case 0: cc = c0; ss = s0; break;
    case 1: cc = -s0; ss = c0; break;
    case 2: cc = -c0; ss = -s0; break;
    default: cc = s0; ss = -c0; break;
  }
  c = cc;
  s = -ss;
}

double mod_wavenumber(int k, int n, double h) {
  const double s = 2.0 * std::sin(M_PI * k / n) / h;
  return s * s;
}

Metric metric_view(const double* mb, const std::vector<size_t>& offs) {
  return Metric{mb + offs[0], mb + offs[1], mb + offs[2], mb + offs[3], mb + offs[4], mb + offs[5],
                mb + offs[6], mb + offs[7], mb + offs[8], mb + offs[9], mb + offs[10], mb + offs[11],
                mb + offs[12]};
}

}  // namespace afid

namespace {

// n = 2^a 3^b 5^c (the radices of the FFT passes)
bool smooth235(int n) {
  if (n <= 0) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

afid_status validate_desc(const afid_grid_desc* d) {
  if (!d || !d->zf) return AFID_ERR_INVALID_ARG;
  if (!smooth235(d->nx) || !smooth235(d->ny) || d->nx % 16 != 0 || d->ny % 8 != 0 || d->nx > 4096 ||
      d->ny > 4096)
    return AFID_ERR_UNSUPPORTED_SIZE;
  if (d->nz < 3 || d->nz > 4096) return AFID_ERR_UNSUPPORTED_SIZE;
  if (!(d->lx > 0.0) || !(d->ly > 0.0)) return AFID_ERR_INVALID_ARG;
  for (int k = 0; k < d->nz; ++k)
    if (!(d->zf[k + 1] > d->zf[k])) return AFID_ERR_INVALID_ARG;
  if (d->precision != AFID_FP64 && d->precision != AFID_MIXED) return AFID_ERR_INVALID_ARG;
  if (d->precision == AFID_MIXED && (d->refine_max_iter < 1 || !(d->refine_tol >= 0.0)))
    return AFID_ERR_INVALID_ARG;
  return AFID_OK;
}

bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

afid_status check_fields(std::initializer_list<const void*> ps) {
  for (const void* p : ps) {
    if (!p) return AFID_ERR_INVALID_ARG;
    if (!aligned(p)) return AFID_ERR_ALIGNMENT;
  }
  return AFID_OK;
}

struct Alloc {
  afid_ctx* c;
  bool ok = true;
  template <typename T> T* get(size_t count) {
    if (!ok || count == 0) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
      ok = false;
      cudaGetLastError();
      return nullptr;
    }
    c->bytes += count * sizeof(T);
    return static_cast<T*>(p);
  }
};

size_t spec_elems(const afid_grid_desc* d) {
  const int M = d->nx / 2;
  const int P = ((M + 1) + 15) / 16 * 16;
  return (size_t)d->nz * d->ny * P;
}

void free_all(afid_ctx* c) {
  void* ps[] = {c->metric_buf, c->twx64, c->twy64, c->ytan64[0], c->ytan64[1], c->xtan64[0], c->xtan64[1], c->twx32, c->twy32, c->mtab64, c->mtab32,
                c->lamx, c->lamy, c->spec, c->phi, c->bbuf, c->R[0], c->R[1], c->R[2],
                c->R[3], c->cntab, c->pa32, c->pc32, c->lowslot, c->low_modes, c->low_scratch, c->scal, c->mtabt32,
                c->part, c->part2, c->part3, c->rres, c->dprev, c->cff, c->stat_buf};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete[] c->zf_host;
  c->zf_host = nullptr;
}

afid_status fill_info(afid_ctx* c, afid_info* info, bool mixed, bool want_div) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFID_ERR_CUDA;
  double s[S_COUNT];
  if (cudaMemcpy(s, c->scal, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return AFID_ERR_CUDA;
  std::memset(info, 0, sizeof(*info));
  if (s[S_FAULT] != 0.0) {
    cudaMemsetAsync(c->scal + S_FAULT, 0, sizeof(double), c->stream);
    return AFID_ERR_TIMEOUT;
  }
  double amax;
  std::memcpy(&amax, &s[S_RHS_ABSMAX], sizeof(double));
  info->rhs_absmax = amax;
  if (mixed) {
    info->iters = (int)s[S_ITERS];
    info->rel_residual = s[S_BNORM2] > 0.0 ? std::sqrt(s[S_RNORM2] / s[S_BNORM2]) : 0.0;  // before the last correction
    info->err_estimate = s[S_ERREST];
    info->rhs_mean = s[S_BMEAN];
  } else {
    info->iters = 1;
    info->rel_residual = 0.0;
    info->rhs_mean = s[S_RHS_MEAN];
  }
  if (want_div) {
    double md;
    std::memcpy(&md, &s[S_MAXDIV], sizeof(double));
    info->max_div = md;
  }
  if (mixed && s[S_CONVERGED] == 0.0) return AFID_ERR_NOT_CONVERGED;
  if (std::fabs(info->rhs_mean) > 1e-8 * info->rhs_absmax && info->rhs_absmax > 0.0)
    return AFID_ERR_INCONSISTENT_RHS;
  return AFID_OK;
}

// Solve L phi = src/s into phi: src = rhs (dev_s = false, s = 1) or D(u, v, w)
// with s from S_PROJ_S. Mixed precision materialises b in bbuf first.
afid_status solve_any(afid_ctx* c, const double* rhs, const double* u, const double* v,
                      const double* w, bool dev_s, double* phi, bool stats) {
  const size_t n = (size_t)c->g.nx * c->g.ny * c->g.nz;
  if (stats && cudaMemsetAsync(c->scal + S_RHS_ABSMAX, 0, sizeof(double), c->stream)) return AFID_ERR_CUDA;
  if (c->prec == AFID_FP64) {
    if (spectral_solve(c, rhs, u, v, w, dev_s, phi, stats)) return AFID_ERR_CUDA;
    return AFID_OK;
  }
  const double* b = rhs;
  if (!rhs) {
    if (divergence_to(c, u, v, w, c->bbuf)) return AFID_ERR_CUDA;
    b = c->bbuf;
  } else if (rhs == phi) {
    if (cudaMemcpyAsync(c->bbuf, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream))
      return AFID_ERR_CUDA;
    b = c->bbuf;
  }
  if (mixed_solve(c, b, phi, stats)) return AFID_ERR_CUDA;
  return AFID_OK;
}

}  // namespace

extern "C" {

const char* afid_status_string(afid_status s) {
  switch (s) {
    case AFID_OK: return "ok";
    case AFID_ERR_INVALID_ARG: return "invalid argument";
    case AFID_ERR_UNSUPPORTED_SIZE:
      return "unsupported grid size (nx, ny of the form 2^a 3^b 5^c, nx a multiple of 16, ny of 8, "
             "both <= 4096; 3 <= nz <= 4096)";
    case AFID_ERR_ALIGNMENT: return "device pointer not 16-byte aligned";
    case AFID_ERR_NOT_CONVERGED: return "mixed-precision refinement did not converge";
    case AFID_ERR_INCONSISTENT_RHS: return "right-hand side has a non-zero weighted mean (removed)";
    case AFID_ERR_CUDA: return "CUDA runtime error";
    case AFID_ERR_OOM: return "device out of memory";
    case AFID_ERR_TIMEOUT: return "a bounded wait inside a kernel timed out (results not valid)";
  }
  return "unknown status";
}

size_t afid_workspace_bytes(const afid_grid_desc* d) {
  if (validate_desc(d) != AFID_OK) return 0;
  const size_t n = (size_t)d->nx * d->ny * d->nz;
  const size_t nf = (size_t)d->nx * d->ny * (d->nz + 1);
  const size_t tab = (size_t)d->nz * (d->ny / 2 + 1) * (d->nx / 2 + 1);
  const bool mixed = d->precision == AFID_MIXED;
  size_t b = spec_elems(d) * (mixed ? 8 : 16) + tab * 8 + (mixed ? tab * 4 : 0);
  b += n * 8;                                   // phi
  if (mixed) b += n * 8 + n * 12;               // kept rhs, residual (two-float), last correction
  if (!(d->flags & AFID_POISSON_ONLY)) b += 2 * n * 8 + 2 * nf * 8;  // R buffers
  return b;
}

afid_status afid_create(const afid_grid_desc* desc, const afid_phys* phys, void* stream,
                        afid_ctx** out) {
  if (!out) return AFID_ERR_INVALID_ARG;
  *out = nullptr;
  afid_status st = validate_desc(desc);
  if (st != AFID_OK) return st;
  afid_ctx* c = new (std::nothrow) afid_ctx;
  if (!c) return AFID_ERR_OOM;
  std::memset(c, 0, sizeof(*c));
  const int nx = desc->nx, ny = desc->ny, nz = desc->nz, M = nx / 2;
  Grid& g = c->g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.M = M;
  g.P = ((M + 1) + 15) / 16 * 16;
  g.nyh = ny / 2 + 1;
  g.dx = desc->lx / nx;
  g.dy = desc->ly / ny;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0 / g.dy;
  g.rdx2 = g.rdx * g.rdx;
  g.rdy2 = g.rdy * g.rdy;
  c->lx = desc->lx;
  c->ly = desc->ly;
  c->prec = desc->precision;
  c->tol = desc->refine_tol;
  c->max_iter = desc->refine_max_iter;
  c->flags = desc->flags;
  if (phys) c->phys = *phys;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return AFID_ERR_CUDA;
  }
  const bool mixed = c->prec == AFID_MIXED;
  // FP64 tridiagonal solver: the warp-partitioned one for long columns and few
  // systems (where one system per thread leaves most of the GPU idle)
  if (c->flags & AFID_WARP_TRIDIAG)
    c->warp_tridiag = 1;
  else if (!(c->flags & AFID_THREAD_TRIDIAG))
    c->warp_tridiag = nz >= 256 && (long long)(M + 1) * ny <= 64LL * c->num_sms;

  c->zf_host = new (std::nothrow) double[nz + 1];
  if (!c->zf_host) {
    delete c;
    return AFID_ERR_OOM;
  }
  std::memcpy(c->zf_host, desc->zf, (nz + 1) * sizeof(double));

  // ---- host metric (wall-normal)
  std::vector<double> flat;
  std::vector<size_t> offs;
  metric_host(nz, g.rdx2, g.rdy2, desc->zf, flat, offs);
  const double* pa = flat.data() + offs[4];
  const double* pc = flat.data() + offs[5];
  const double* pdiag = flat.data() + offs[12];
  c->hz = 0.0;
  for (int k = 0; k < nz; ++k) c->hz += flat[offs[0] + k];  // the order the kernels summed in

  // ---- host tables
  std::vector<double2> twx(nx), twy(ny);
  std::vector<float2> twx32(nx), twy32(ny);
  for (int m = 0; m < nx; ++m) {
    twiddle(m, nx, twx[m].x, twx[m].y);
    twx32[m] = make_float2((float)twx[m].x, (float)twx[m].y);
  }
  for (int m = 0; m < ny; ++m) {
    twiddle(m, ny, twy[m].x, twy[m].y);
    twy32[m] = make_float2((float)twy[m].x, (float)twy[m].y);
  }
  std::vector<double> lamx(M + 1), lamy(g.nyh);
  for (int k = 0; k <= M; ++k) lamx[k] = mod_wavenumber(k, nx, g.dx);
  for (int k = 0; k < g.nyh; ++k) lamy[k] = mod_wavenumber(k, ny, g.dy);
  std::vector<int> lowslot;
  std::vector<int2> low;
  if (mixed) {
    const double lmin = std::fmin(lamx[1], lamy[1]);
    c->lam_thr = 64.0 * lmin;
    lowslot.assign((size_t)ny * (M + 1), -1);
    for (int ky = 0; ky < ny; ++ky) {
      const int kyh = ky < ny - ky ? ky : ny - ky;
      for (int kx = 0; kx <= M; ++kx) {
        if (kx == 0 && ky == 0) continue;
        if (lamx[kx] + lamy[kyh] < c->lam_thr) {
          lowslot[(size_t)ky * (M + 1) + kx] = c->nlow++;
          low.push_back(make_int2(ky, kx));
        }
      }
    }
  }

  // ---- device allocations
  Alloc A{c};
  const size_t n = (size_t)nx * ny * nz, nf = (size_t)nx * ny * (nz + 1);
  const size_t tab = (size_t)nz * g.nyh * (M + 1);
  c->metric_buf = A.get<double>(flat.size());
  c->twx64 = A.get<double2>(nx);
  c->twy64 = A.get<double2>(ny);
  // tangent-form tables of the FP64 y transform (power-of-two ny >= 64)
  // (the tile of the y kernel then has at most 512 threads: ny <= 4096)
  const bool ytan = ny >= 64 && ny <= 4096 && (ny & (ny - 1)) == 0;
  c->ytan_len = ytan ? tan_tables(ny, nullptr, false, nullptr) : 0;
  if (ytan) {
    c->ytan64[0] = A.get<double>(c->ytan_len);
    c->ytan64[1] = A.get<double>(c->ytan_len);
  }
  const bool xtan = M >= 64 && (M & (M - 1)) == 0;
  c->xtan_len = xtan ? tan_tables(M, nullptr, false, nullptr) : 0;
  if (xtan) {
    c->xtan64[0] = A.get<double>(c->xtan_len);
    c->xtan64[1] = A.get<double>(c->xtan_len);
  }
  c->twx32 = A.get<float2>(nx);
  c->twy32 = A.get<float2>(ny);
  c->lamx = A.get<double>(M + 1);
  c->lamy = A.get<double>(g.nyh);
  c->mtab64 = A.get<double>(tab);
  if (mixed) c->mtab32 = A.get<float>(tab);
  const size_t se = (size_t)nz * ny * g.P;
  c->spec = mixed ? (void*)A.get<float2>(se) : (void*)A.get<double2>(se);
  c->phi = A.get<double>(n);
  if (mixed) {
    c->bbuf = A.get<double>(n);
    c->rres = A.get<float2>(n);
    c->dprev = A.get<float>(n);
    c->cff = A.get<float2>((size_t)3 * nz);
    c->pa32 = A.get<float>(nz);
    c->pc32 = A.get<float>(nz);
    c->lowslot = A.get<int>((size_t)ny * (M + 1));
    if (c->nlow) c->low_modes = A.get<int2>(c->nlow);
    std::vector<int> per_col(M + 1, 0);  // low modes per kx column
    for (const int2& md : low) per_col[md.y]++;
    int lmax = 0;
    for (int v : per_col) lmax = v > lmax ? v : lmax;
    if (init_yfft_thomas32(c, lmax) == cudaSuccess && c->fuse_yt)  // small nz: fused kernel's table
      c->mtabt32 = A.get<float>(tab);
  }
  if (!(c->flags & AFID_POISSON_ONLY)) {
    c->R[0] = A.get<double>(n);
    c->R[1] = A.get<double>(n);
    c->R[2] = A.get<double>(nf);
    c->R[3] = A.get<double>(nf);
  }
  c->cntab = A.get<double>((size_t)3 * CN_TAB_ARRAYS * (nz + 1));
  c->scal = A.get<double>(S_COUNT);
  c->stat_buf = A.get<double>((size_t)(nz + 1) * AFID_STAT_NQ + 8);
  c->part_len = c->num_sms * 8;
  c->part = A.get<double>((size_t)3 * c->part_len);
  if (mixed) {
    c->part2_len = c2r_blocks(g);
    c->part2 = A.get<double>((size_t)2 * c->part2_len);
    c->part3 = A.get<double>((size_t)3 * c->part2_len);
  }
  if (!A.ok) {
    free_all(c);
    delete c;
    return AFID_ERR_OOM;
  }
  c->m = metric_view(static_cast<const double*>(c->metric_buf), offs);
  bool ok = true;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (dst && bytes) ok = ok && cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  up(c->metric_buf, flat.data(), flat.size() * sizeof(double));
  up(c->twx64, twx.data(), nx * sizeof(double2));
  up(c->twy64, twy.data(), ny * sizeof(double2));
  if (c->ytan_len > 0) {
    std::vector<double> tt(c->ytan_len);
    for (int d = 0; d < 2; ++d) {
      tan_tables(ny, twy.data(), d == 1, tt.data());
      up(c->ytan64[d], tt.data(), tt.size() * sizeof(double));
    }
  }
  if (c->xtan_len > 0) {
    std::vector<double2> twm(M);  // exp(-2 pi i m/M) = the x table at even indices
    for (int q = 0; q < M; ++q) twm[q] = twx[2 * q];
    std::vector<double> tt(c->xtan_len);
    for (int d = 0; d < 2; ++d) {
      tan_tables(M, twm.data(), d == 1, tt.data());
      up(c->xtan64[d], tt.data(), tt.size() * sizeof(double));
    }
  }
  up(c->twx32, twx32.data(), nx * sizeof(float2));
  up(c->twy32, twy32.data(), ny * sizeof(float2));
  up(c->lamx, lamx.data(), (M + 1) * sizeof(double));
  up(c->lamy, lamy.data(), g.nyh * sizeof(double));
  if (mixed) {
    std::vector<float> pa32(nz), pc32(nz);
    for (int k = 0; k < nz; ++k) {
      pa32[k] = (float)pa[k];
      pc32[k] = (float)pc[k];
    }
    up(c->pa32, pa32.data(), nz * sizeof(float));
    up(c->pc32, pc32.data(), nz * sizeof(float));
    // two-float splits (head = nearest FP32, tail = FP32 of the remainder) of
    // pa, pc, pdiag for the extended-precision residual update
    std::vector<float2> cff((size_t)3 * nz);
    auto split = [](double x) {
      const float h = (float)x;
      return make_float2(h, (float)(x - (double)h));
    };
    for (int k = 0; k < nz; ++k) {
      cff[k] = split(pa[k]);
      cff[nz + k] = split(pc[k]);
      cff[2 * nz + k] = split(pdiag[k]);
    }
    up(c->cff, cff.data(), cff.size() * sizeof(float2));
    up(c->lowslot, lowslot.data(), lowslot.size() * sizeof(int));
    if (c->nlow) up(c->low_modes, low.data(), low.size() * sizeof(int2));
  }
  ok = ok && cudaMemset(c->spec, 0, se * (mixed ? sizeof(float2) : sizeof(double2))) == cudaSuccess;
  ok = ok && cudaMemset(c->scal, 0, S_COUNT * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMemset(c->cntab, 0, (size_t)3 * CN_TAB_ARRAYS * (nz + 1) * sizeof(double)) == cudaSuccess;
  ok = ok && init_thomas_tables(c) == cudaSuccess;
  ok = ok && ((c->flags & AFID_NO_TMA) || init_ffty_tma(c) == cudaSuccess);
  ok = ok && cudaStreamSynchronize(c->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return AFID_ERR_CUDA;
  }
  *out = c;
  return AFID_OK;
}

afid_status afid_destroy(afid_ctx* c) {
  if (!c) return AFID_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  if (c->prof) {
    for (cudaEvent_t e : c->prof->ev) cudaEventDestroy(e);
    delete c->prof;
  }
  free_all(c);
  delete c;
  return AFID_OK;
}

afid_status afid_set_stream(afid_ctx* c, void* stream) {
  if (!c) return AFID_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return AFID_OK;
}

long long afid_kernel_launches(const afid_ctx* c) { return c ? c->launches : -1; }

afid_status afid_profile_enable(afid_ctx* c, int on) {
  if (!c) return AFID_ERR_INVALID_ARG;
  if (!c->prof) {
    c->prof = new (std::nothrow) Prof;
    if (!c->prof) return AFID_ERR_OOM;
    const int n = 1 << 15;
    c->prof->ev.resize(n);
    c->prof->fam.resize(n / 2);
    for (int i = 0; i < n; ++i)
      if (cudaEventCreate(&c->prof->ev[i]) != cudaSuccess) return AFID_ERR_CUDA;
  }
  c->prof->on = on != 0;
  return AFID_OK;
}

afid_status afid_profile_read(afid_ctx* c, double* ms, long long* launches, int n) {
  if (!c || !c->prof || n < 0) return AFID_ERR_INVALID_ARG;
  Prof* p = c->prof;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFID_ERR_CUDA;
  for (int i = 0; i + 1 < p->used; i += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]) != cudaSuccess) return AFID_ERR_CUDA;
    p->ms[p->fam[i / 2]] += t;
    p->n[p->fam[i / 2]] += 1;
  }
  p->used = 0;
  for (int f = 0; f < n && f < KF_COUNT; ++f) {
    if (ms) ms[f] = p->ms[f];
    if (launches) launches[f] = p->n[f];
    p->ms[f] = 0.0;
    p->n[f] = 0;
  }
  const bool of = p->overflow;
  p->overflow = false;
  return of ? AFID_ERR_INVALID_ARG : AFID_OK;
}

const char* afid_kernel_family_name(int f) {
  static const char* names[] = {"r2c_x", "fft_y", "thomas", "zero_mode", "c2r_x", "project",
                                "rhs", "crank_nicolson", "cfl_reduce", "refine", "adjoint",
                                "cn_tables", "mr_prolong", "mr_scalar_rhs", "mr_restrict",
                                "yfft_thomas"};
  return (f >= 0 && f < KF_COUNT) ? names[f] : "unknown";
}

afid_status afid_poisson_solve(afid_ctx* c, const double* rhs, double* phi, afid_info* info) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({rhs, phi});
  if (st) return st;
  st = solve_any(c, rhs, nullptr, nullptr, nullptr, false, phi, info != nullptr);
  if (st) return st;
  if (cudaGetLastError() != cudaSuccess) return AFID_ERR_CUDA;
  return info ? fill_info(c, info, c->prec == AFID_MIXED, false) : AFID_OK;
}

afid_status afid_project(afid_ctx* c, double* u, double* v, double* w, double* p, double s,
                         double beta, afid_info* info) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({u, v, w, p});
  if (st) return st;
  if (!(s > 0.0) || !std::isfinite(beta)) return AFID_ERR_INVALID_ARG;
  if (set_proj_scalars(c, s, beta)) return AFID_ERR_CUDA;
  st = solve_any(c, nullptr, u, v, w, true, c->phi, info != nullptr);
  if (st) return st;
  if (project(c, u, v, w, p, c->phi)) return AFID_ERR_CUDA;
  if (info) {
    if (max_divergence(c, u, v, w, c->scal + S_MAXDIV)) return AFID_ERR_CUDA;
    return fill_info(c, info, c->prec == AFID_MIXED, true);
  }
  return cudaGetLastError() == cudaSuccess ? AFID_OK : AFID_ERR_CUDA;
}

afid_status afid_cfl(afid_ctx* c, const double* u, const double* v, const double* w, double cflv,
                     double dt_max, double* cflm_dev) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({u, v, w});
  if (st) return st;
  if (!(cflv > 0.0) || !(dt_max > 0.0)) return AFID_ERR_INVALID_ARG;
  if (cflm_dev && !aligned(cflm_dev) && (reinterpret_cast<uintptr_t>(cflm_dev) & 7u)) return AFID_ERR_ALIGNMENT;
  return cfl(c, u, v, w, cflv, dt_max, cflm_dev) ? AFID_ERR_CUDA : AFID_OK;
}

afid_status afid_max_divergence(afid_ctx* c, const double* u, const double* v, const double* w,
                                double* out_dev) {
  if (!c || !out_dev || (reinterpret_cast<uintptr_t>(out_dev) & 7u)) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({u, v, w});
  if (st) return st;
  return max_divergence(c, u, v, w, out_dev) ? AFID_ERR_CUDA : AFID_OK;
}

afid_status afid_rk3_substep(afid_ctx* c, int l, double dt, double* u, double* v, double* w,
                             double* T, double* p, double* Hu, double* Hv, double* Hw, double* HT,
                             afid_info* info) {
  if (!c) return AFID_ERR_INVALID_ARG;
  if (c->flags & AFID_POISSON_ONLY) return AFID_ERR_INVALID_ARG;
  if (l < 0 || l > 2 || !std::isfinite(dt)) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({u, v, w, p, Hu, Hv, Hw});
  if (st) return st;
  if (HT && !T) return AFID_ERR_INVALID_ARG;
  if (T && (st = check_fields({T}))) return st;
  if (HT && (st = check_fields({HT}))) return st;
  if (cn_tables(c, l, dt)) return AFID_ERR_CUDA;
  if (rk3_explicit(c, l, dt, u, v, w, T, p, Hu, Hv, Hw, HT)) return AFID_ERR_CUDA;
  if (cn_sweeps(c, u, v, w, HT ? T : nullptr)) return AFID_ERR_CUDA;
  st = solve_any(c, nullptr, u, v, w, true, c->phi, info != nullptr);
  if (st) return st;
  if (project(c, u, v, w, p, c->phi)) return AFID_ERR_CUDA;
  if (info) {
    if (max_divergence(c, u, v, w, c->scal + S_MAXDIV)) return AFID_ERR_CUDA;
    return fill_info(c, info, c->prec == AFID_MIXED, true);
  }
  return cudaGetLastError() == cudaSuccess ? AFID_OK : AFID_ERR_CUDA;
}

afid_status afid_statistics(afid_ctx* c, const double* u, const double* v, const double* w,
                            const double* T, double* profiles, afid_stats* out) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({u, v, w});
  if (st) return st;
  if (T && (st = check_fields({T}))) return st;
  if (statistics(c, u, v, w, T)) return AFID_ERR_CUDA;
  const size_t np = (size_t)(c->g.nz + 1) * AFID_STAT_NQ;
  double sc[8];
  if (profiles &&
      cudaMemcpyAsync(profiles, c->stat_buf, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream))
    return AFID_ERR_CUDA;
  if (cudaMemcpyAsync(sc, c->stat_buf + np, sizeof(sc), cudaMemcpyDeviceToHost, c->stream))
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

afid_status afid_nusselt(afid_ctx* c, const double* w, const double* T, double coef,
                         double* nu_out, double* gw, double* gT) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({w, T});
  if (st) return st;
  if (gw && !aligned(gw)) return AFID_ERR_ALIGNMENT;
  if (gT && !aligned(gT)) return AFID_ERR_ALIGNMENT;
  if (!std::isfinite(coef)) return AFID_ERR_INVALID_ARG;
  if (nusselt(c, w, T, coef, gw, gT)) return AFID_ERR_CUDA;
  if (nu_out) {
    if (cudaMemcpyAsync(nu_out, c->stat_buf + (c->g.nz + 1), sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream))
      return AFID_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream)) return AFID_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? AFID_OK : AFID_ERR_CUDA;
}

afid_status afid_poisson_solve_adjoint(afid_ctx* c, const double* gphi, double* grhs) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({gphi, grhs});
  if (st) return st;
  // solve^T y = W_c solve(W_c^-1 y)
  if (scale_cells(c, gphi, grhs, false)) return AFID_ERR_CUDA;
  if ((st = solve_any(c, grhs, nullptr, nullptr, nullptr, false, grhs, false))) return st;
  if (scale_cells(c, grhs, grhs, true)) return AFID_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? AFID_OK : AFID_ERR_CUDA;
}

static afid_status projection_adjoint(afid_ctx* c, double* gu, double* gv, double* gw, double* gp) {
  if (project_adjoint_pre(c, gu, gv, gw, gp, 0.0, 0.0)) return AFID_ERR_CUDA;
  afid_status st = solve_any(c, c->phi, nullptr, nullptr, nullptr, false, c->phi, false);
  if (st) return st;
  if (project_adjoint_post(c, gu, gv, gw, gp, c->phi, 0.0, 0.0)) return AFID_ERR_CUDA;
  return AFID_OK;
}

afid_status afid_project_adjoint(afid_ctx* c, double* gu, double* gv, double* gw, double* gp,
                                 double s, double beta) {
  if (!c) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({gu, gv, gw, gp});
  if (st) return st;
  if (!(s > 0.0) || !std::isfinite(beta)) return AFID_ERR_INVALID_ARG;
  if (set_proj_scalars(c, s, beta)) return AFID_ERR_CUDA;
  if ((st = projection_adjoint(c, gu, gv, gw, gp))) return st;
  return cudaGetLastError() == cudaSuccess ? AFID_OK : AFID_ERR_CUDA;
}

afid_status afid_rk3_substep_adjoint(afid_ctx* c, int l, double dt, const double* u,
                                     const double* v, const double* w, const double* T,
                                     double* gu, double* gv, double* gw, double* gT, double* gp,
                                     double* gHu, double* gHv, double* gHw, double* gHT) {
  if (!c) return AFID_ERR_INVALID_ARG;
  if (c->flags & AFID_POISSON_ONLY) return AFID_ERR_INVALID_ARG;
  if (l < 0 || l > 2 || !(dt > 0.0)) return AFID_ERR_INVALID_ARG;
  afid_status st = check_fields({u, v, w, gu, gv, gw, gp, gHu, gHv, gHw});
  if (st) return st;
  if ((T == nullptr) != (gT == nullptr) || (T == nullptr) != (gHT == nullptr)) return AFID_ERR_INVALID_ARG;
  if (T && (st = check_fields({T, gT, gHT}))) return st;
  // reverse order of the forward substep: projection, Crank-Nicolson, explicit terms
  if (cn_tables(c, l, dt)) return AFID_ERR_CUDA;
  if ((st = projection_adjoint(c, gu, gv, gw, gp))) return st;
  if (cn_sweeps_adjoint(c, gu, gv, gw, gT)) return AFID_ERR_CUDA;
  if (adjoint_explicit(c, l, dt, u, v, w, T, gu, gv, gw, gT, gp, gHu, gHv, gHw, gHT))
    return AFID_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? AFID_OK : AFID_ERR_CUDA;
}

}  // extern "C"
