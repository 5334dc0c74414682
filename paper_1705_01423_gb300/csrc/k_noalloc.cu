// Poisson solve without any device allocation: every piece of workspace (the
// metric, twiddles, wavenumbers, the reciprocal-pivot table and the spectral
// array) lives in one file-scope __device__ array of fixed size, so callers
// that cannot call cudaMalloc (code running under an allocator it does not
// own, a real-time loop that must not allocate, a plugin with no context
// object) can still solve. The arithmetic is that of afid_poisson_solve in
// AFID_FP64: the same kernels run on the same host-computed tables.
#include <cmath>
#include <cstring>
#include <mutex>

#include "afid_internal.cuh"

using namespace afid;

namespace {

constexpr size_t kNoallocBytes = (size_t)16 << 20;  // 16 MiB per device
__device__ __align__(256) unsigned char g_noalloc_ws[kNoallocBytes];

constexpr int kMaxDevices = 64;
void* g_ws_addr[kMaxDevices] = {};  // device address of g_noalloc_ws, per device
std::mutex g_mu;                    // guards g_ws_addr and the host staging buffer

// Host staging for the tables uploaded on every call (no heap allocation).
constexpr int kMaxN = 4096;
double g_stage[13 * (kMaxN + 1) + 2 * (2 * kMaxN) + 2 * (kMaxN / 2 + 1)];

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

struct Layout {
  size_t metric, twx, twy, lamx, lamy, scal, mtab, spec, total;
};

Layout layout(int nx, int ny, int nz) {
  const int M = nx / 2, P = ((M + 1) + 15) / 16 * 16, nyh = ny / 2 + 1;
  Layout L;
  size_t o = 0;
  L.metric = o;
  o += up256((size_t)13 * (nz + 1) * sizeof(double));
  L.twx = o;
  o += up256((size_t)nx * sizeof(double2));
  L.twy = o;
  o += up256((size_t)ny * sizeof(double2));
  L.lamx = o;
  o += up256((size_t)(M + 1) * sizeof(double));
  L.lamy = o;
  o += up256((size_t)nyh * sizeof(double));
  L.scal = o;
  o += up256((size_t)S_COUNT * sizeof(double));
  L.mtab = o;
  o += up256((size_t)nz * nyh * (M + 1) * sizeof(double));
  L.spec = o;
  o += up256((size_t)nz * ny * P * sizeof(double2));
  L.total = o;
  return L;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

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
  if (r == 0) {
    c0 = 1.0;
    s0 = 0.0;
  }
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

}  // namespace

extern "C" afid_status afid_poisson_solve_noalloc(int nx, int ny, int nz, double lx, double ly,
                                                  const double* zf, const double* rhs, double* phi,
                                                  void* stream) {
  if (!zf || !rhs || !phi) return AFID_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(rhs) & 15u) || (reinterpret_cast<uintptr_t>(phi) & 15u))
    return AFID_ERR_ALIGNMENT;
  if (!pow2(nx) || !pow2(ny) || nx < 16 || ny < 8 || nx > kMaxN || ny > kMaxN || nz < 3 || nz > kMaxN)
    return AFID_ERR_UNSUPPORTED_SIZE;
  if (!(lx > 0.0) || !(ly > 0.0)) return AFID_ERR_INVALID_ARG;
  for (int k = 0; k < nz; ++k)
    if (!(zf[k + 1] > zf[k])) return AFID_ERR_INVALID_ARG;
  const Layout L = layout(nx, ny, nz);
  if (L.total > kNoallocBytes) return AFID_ERR_UNSUPPORTED_SIZE;  // grid too large for the fixed workspace

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AFID_ERR_CUDA;
  if (!g_ws_addr[dev]) {  // once per device, with that device current
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) {
      cudaGetLastError();
      return AFID_ERR_CUDA;
    }
    g_ws_addr[dev] = p;
  }
  unsigned char* ws = static_cast<unsigned char*>(g_ws_addr[dev]);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // ---- host tables, same formulas as afid_create
  afid_ctx c;
  std::memset(&c, 0, sizeof(c));
  Grid& g = c.g;
  const int M = nx / 2;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.M = M;
  g.P = ((M + 1) + 15) / 16 * 16;
  g.nyh = ny / 2 + 1;
  g.dx = lx / nx;
  g.dy = ly / ny;
  g.rdx = 1.0 / g.dx;
  g.rdy = 1.0 / g.dy;
  g.rdx2 = g.rdx * g.rdx;
  g.rdy2 = g.rdy * g.rdy;
  const int Lz = nz + 1;
  double* h = g_stage;
  double *dzc = h, *rdzc = h + Lz, *dzf = h + 2 * Lz, *rdzf = h + 3 * Lz, *pa = h + 4 * Lz,
         *pc = h + 5 * Lz, *ca = h + 6 * Lz, *cc = h + 7 * Lz, *fa = h + 8 * Lz, *fc = h + 9 * Lz,
         *wlo = h + 10 * Lz, *whi = h + 11 * Lz, *pdiag = h + 12 * Lz;
  std::memset(h, 0, sizeof(double) * 13 * Lz);
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
    pdiag[k] = pa[k] + pc[k] + 2.0 * g.rdx2 + 2.0 * g.rdy2;
  }
  for (int k = 1; k < nz; ++k) {
    fa[k] = 1.0 / (dzf[k] * dzc[k - 1]);
    fc[k] = 1.0 / (dzf[k] * dzc[k]);
    wlo[k] = dzc[k - 1] / (2.0 * dzf[k]);
    whi[k] = dzc[k] / (2.0 * dzf[k]);
  }
  double* tw = h + 13 * Lz;  // nx + ny complex
  for (int m = 0; m < nx; ++m) twiddle(m, nx, tw[2 * m], tw[2 * m + 1]);
  double* twy = tw + 2 * nx;
  for (int m = 0; m < ny; ++m) twiddle(m, ny, twy[2 * m], twy[2 * m + 1]);
  double* lam = twy + 2 * ny;  // M+1 then nyh
  for (int k = 0; k <= M; ++k) {
    const double s = 2.0 * std::sin(M_PI * k / nx) / g.dx;
    lam[k] = s * s;
  }
  for (int k = 0; k < g.nyh; ++k) {
    const double s = 2.0 * std::sin(M_PI * k / ny) / g.dy;
    lam[M + 1 + k] = s * s;
  }

  // ---- device views into the fixed workspace
  const double* mb = reinterpret_cast<const double*>(ws + L.metric);
  c.m = Metric{mb, mb + Lz, mb + 2 * Lz, mb + 3 * Lz, mb + 4 * Lz, mb + 5 * Lz, mb + 6 * Lz,
               mb + 7 * Lz, mb + 8 * Lz, mb + 9 * Lz, mb + 10 * Lz, mb + 11 * Lz, mb + 12 * Lz};
  c.twx64 = reinterpret_cast<double2*>(ws + L.twx);
  c.twy64 = reinterpret_cast<double2*>(ws + L.twy);
  c.lamx = reinterpret_cast<double*>(ws + L.lamx);
  c.lamy = reinterpret_cast<double*>(ws + L.lamy);
  c.scal = reinterpret_cast<double*>(ws + L.scal);
  c.mtab64 = reinterpret_cast<double*>(ws + L.mtab);
  c.spec = ws + L.spec;
  c.prec = AFID_FP64;
  c.stream = st;
  c.device = dev;

  bool ok = true;
  ok = ok && cudaMemcpyAsync(ws + L.metric, h, sizeof(double) * 13 * Lz, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(ws + L.twx, tw, sizeof(double2) * nx, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(ws + L.twy, twy, sizeof(double2) * ny, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(ws + L.lamx, lam, sizeof(double) * (M + 1), cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(ws + L.lamy, lam + M + 1, sizeof(double) * g.nyh, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(ws + L.scal, 0, sizeof(double) * S_COUNT, st) == cudaSuccess;
  // copies from pageable host memory return once the data has left g_stage,
  // so the staging buffer can be refilled by the next call
  ok = ok && init_thomas_tables(&c) == cudaSuccess;
  ok = ok && spectral_solve(&c, rhs, nullptr, nullptr, nullptr, false, phi, false) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return AFID_ERR_CUDA;
  }
  return AFID_OK;
}
