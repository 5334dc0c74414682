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

std::mutex g_mu;  // serialises host callers: guards the host staging buffer

// Host staging for the tables uploaded on every call (no heap allocation).
constexpr int kMaxN = 4096;
double g_stage[METRIC_ARRAYS * (kMaxN + 1) + 2 * (2 * kMaxN) + 2 * (kMaxN / 2 + 1)];

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

struct Layout {
  size_t metric, twx, twy, lamx, lamy, scal, mtab, spec, total;
};

Layout layout(int nx, int ny, int nz) {
  const int M = nx / 2, P = ((M + 1) + 15) / 16 * 16, nyh = ny / 2 + 1;
  Layout L;
  size_t o = 0;
  L.metric = o;
  o += up256((size_t)METRIC_ARRAYS * (nz + 1) * sizeof(double));
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
  if (cudaGetDevice(&dev) != cudaSuccess) return AFID_ERR_CUDA;
  // The array's device address, looked up on every call for the device and
  // context current now (no allocation): an address cached from an earlier
  // call could belong to another context of the same device, or to a context
  // destroyed since by cudaDeviceReset, where the module is loaded again at
  // another address. The first call on a device also loads the library's
  // device code there.
  void* wsp = nullptr;
  if (cudaGetSymbolAddress(&wsp, g_noalloc_ws) != cudaSuccess || !wsp) {
    cudaGetLastError();
    return AFID_ERR_CUDA;
  }
  unsigned char* ws = static_cast<unsigned char*>(wsp);
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
  metric_fill(nz, g.rdx2, g.rdy2, zf, h);  // the arrays of Metric, each nz+1 long
  double* tw = h + METRIC_ARRAYS * Lz;  // nx + ny complex
  for (int m = 0; m < nx; ++m) twiddle(m, nx, tw[2 * m], tw[2 * m + 1]);
  double* twy = tw + 2 * nx;
  for (int m = 0; m < ny; ++m) twiddle(m, ny, twy[2 * m], twy[2 * m + 1]);
  double* lam = twy + 2 * ny;  // M+1 then nyh
  for (int k = 0; k <= M; ++k) lam[k] = mod_wavenumber(k, nx, g.dx);
  for (int k = 0; k < g.nyh; ++k) lam[M + 1 + k] = mod_wavenumber(k, ny, g.dy);

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
  ok = ok && cudaMemcpyAsync(ws + L.metric, h, sizeof(double) * METRIC_ARRAYS * Lz, cudaMemcpyHostToDevice, st) == cudaSuccess;
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
