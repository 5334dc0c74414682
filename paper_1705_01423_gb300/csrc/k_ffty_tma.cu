// Complex FFT along y (Sec. 2.2, the second of the two periodic transforms)
// with TMA-staged tiles: the on-device replacement of the paper's y-pencil
// transpose (Sec. 3.5).
//
// The spectral array [nz][ny][P] (complex, row pitch P) is read as a 3-D
// tensor of scalars {2 (M + 1), ny, nz}. One tile is TK consecutive kx
// columns x all ny rows of one z plane; its box lands in shared memory as
// rows of TK complex values, so that the TK lines are transformed side by
// side: the lanes of a warp run along kx and every Stockham access reads or
// writes whole rows. TK = 16 (128-byte rows) up to ny = 512; beyond, TK =
// 8192 / ny (8 at 1024, 4 at 2048: 64- and 32-byte rows, still whole DRAM
// sectors), which keeps a stage at 64 KB and the block at ny/8 threads per
// line = 1024. Columns beyond kx = M are outside the tensor: they load as
// zeros and are not stored.
//
// A persistent block walks its tiles with a ring of S shared-memory stages:
// while tile i is transformed, the load of tile i+1 and the store of tile i-1
// are in flight (one mbarrier per stage for loads, bulk groups for stores).
// Waits are bounded (2 s); a timeout sets the device flag S_FAULT and the block
// stops after waiting (again bounded) for its own copies in flight. A test
// hook (afid_test_tma_timeout) makes one launch's block 0 arm a stage without
// issuing its copy, under a 1 ms limit, so that this path runs without any
// fault or hang.
#include "afid_internal.cuh"
#include "fft.cuh"
#include "tma.cuh"

namespace afid {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Used for the FP32 transforms of the mixed-precision solve, which are bound
// by HBM bandwidth. The FP64 transforms stay on the plain kernel: they are
// bound by the FP64 issue rate, and there two 512-thread blocks per SM of the
// plain kernel keep the FP64 pipe busier than one block of this ring (whose
// 64 KB stages allow one block per SM at ny = 512); measured at 512 x 512 x
// 384, 5.08 ms (plain) against 5.46 ms (ring) for the two y passes of a solve.
// TK columns per tile; the block has TK x ny/8 <= 1024 threads
constexpr int kTmaMaxThreads = 1024;
inline int tma_tile_columns(int ny) { return ny <= 512 ? 16 : 8192 / ny; }

template <typename R, bool INV, int TK>
__global__ void __launch_bounds__(kTmaMaxThreads, 1) k_fft_y_tma(const __grid_constant__ CUtensorMap map, Grid g,
                                                       const typename cplx<R>::T* __restrict__ tw,
                                                       const double* __restrict__ skip,
                                                       double* __restrict__ scal, int stages,
                                                       int ntile_x, int stall_block, uint64_t limit_ns) {
  using C = typename cplx<R>::T;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int N = g.ny;
  const int tile_elems = TK * N;
  C* tiles = reinterpret_cast<C*>(smem_raw);
  C* stw = tiles + (size_t)stages * tile_elems;
  uint64_t* bar = reinterpret_cast<uint64_t*>(stw + N);
  const int tid = threadIdx.x;
  const int BR = N < 256 ? N : 256;  // rows per box (box extents are <= 256)
  const uint32_t tile_bytes = (uint32_t)(tile_elems * sizeof(C));
  const int ntiles = ntile_x * g.nz;
  const int first = blockIdx.x;
  const int count = first < ntiles ? (ntiles - 1 - first) / gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  // per-pass twiddle tables (N - 1 entries): the lanes of a warp hold 32 / TK
  // consecutive butterflies, whose twiddles in the table of length N lie
  // r k N/(p R) apart (up to 8-way bank conflicts at TK = 4)
  pass_twiddles(stw, tw, N, 1, tid, blockDim.x);
  __syncthreads();

  // thread 0: start the loads of local tile `it` into stage it % stages. The
  // block numbered stall_block (a test of the timeout path; -1 otherwise) arms
  // its first stage with the tile's byte count and issues no copy, so that its
  // wait runs out with nothing in flight for that stage.
  auto issue = [&](int it) {
    const int tile = first + it * gridDim.x;
    const int s = it % stages;
    const int kxt = tile % ntile_x, z = tile / ntile_x;
    mbar_expect_tx(&bar[s], tile_bytes);
    if (it == 0 && (int)blockIdx.x == stall_block) return;
    for (int y0 = 0; y0 < N; y0 += BR)
      tma_load_3d(tiles + (size_t)s * tile_elems + (size_t)y0 * TK, &map, &bar[s], 2 * kxt * TK, y0, z);
  };
  if (tid == 0 && count > 0) issue(0);

  const int c = tid % TK, t = tid / TK;  // column within the tile, thread within the line
  bool failed = false;
  int it = 0;
  for (; it < count; ++it) {
    const int s = it % stages;
    if (tid == 0 && it + 1 < count) {
      // stage (it+1) % stages last held tile it+1-stages: its store must have
      // finished reading shared memory before the next load overwrites it
      if (stages >= 3) bulk_wait_read<1>();
      else bulk_wait_read<0>();
      issue(it + 1);
    }
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((it / stages) & 1), limit_ns);
    if (__syncthreads_or(!ok)) {  // block-uniform decision
      failed = true;
      break;
    }
    C* buf = tiles + (size_t)s * tile_elems;
    fft_line_pt_ix<INV, TK == 4 ? 3 : (TK == 8 ? 1 : 0)>(buf, N, stw, t, true, ColIx<TK>{c});
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      const int tile = first + it * gridDim.x;
      const int kxt = tile % ntile_x, z = tile / ntile_x;
      for (int y0 = 0; y0 < N; y0 += BR) tma_store_3d(&map, buf + (size_t)y0 * TK, 2 * kxt * TK, y0, z);
      bulk_commit();
    }
  }
  if (tid == 0) {
    if (failed) {
      scal[S_FAULT] = 1.0;
      // loads of tiles it and it+1 may still be in flight: wait for them (bounded)
      for (int q = it; q < count && q <= it + 1; ++q)
        mbar_wait_bounded(&bar[q % stages], (uint32_t)((q / stages) & 1), limit_ns);
    }
    bulk_wait<0>();  // every store complete before the block's shared memory is released
  }
}

// Host: tensor map of the spectral workspace for the y transforms.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && p)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

template <typename R>
static size_t ffty_tma_smem(const Grid& g, int TK, int stages) {
  using C = typename cplx<R>::T;
  return (size_t)stages * TK * g.ny * sizeof(C) + (size_t)g.ny * sizeof(C) + stages * sizeof(uint64_t);
}

template <bool INV>
static void* tma_kernel(int TK) {
  return TK == 16 ? (void*)k_fft_y_tma<float, INV, 16>
                  : (TK == 8 ? (void*)k_fft_y_tma<float, INV, 8> : (void*)k_fft_y_tma<float, INV, 4>);
}

// Sets up the TMA y transform of a mixed-precision context when the sizes
// allow it (ny a power of two, 16 <= ny <= 2048, a tile ring of at least two
// stages in shared memory); leaves c->tma_y = 0 (the plain kernel is used)
// otherwise.
cudaError_t init_ffty_tma(afid_ctx* c) {
  c->tma_y = 0;
  const Grid& g = c->g;
  if (g.ny > 2048 || g.ny < 8 || (g.ny & (g.ny - 1)) != 0) return cudaSuccess;  // power-of-two ny
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaSuccess;
  if (c->prec != AFID_MIXED) return cudaSuccess;
  const int TK = tma_tile_columns(g.ny);
  const size_t csz = sizeof(float2);
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  int stages = 3;
  auto need = [&](int s) { return ffty_tma_smem<float>(g, TK, s); };
  // + static shared memory of the kernel (128 B)
  while (stages > 2 && need(stages) + 256 > (size_t)smem_optin) --stages;
  if (need(stages) + 256 > (size_t)smem_optin) return cudaSuccess;
  const int threads = TK * (g.ny / 8);
  if (threads > kTmaMaxThreads || threads < 32) return cudaSuccess;

  cuuint64_t dims[3] = {(cuuint64_t)2 * (g.M + 1), (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)g.P * csz, (cuuint64_t)g.ny * g.P * csz};
  cuuint32_t box[3] = {(cuuint32_t)(2 * TK), (cuuint32_t)(g.ny < 256 ? g.ny : 256), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(&c->tmy, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                   c->spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaSuccess;
  const size_t sm = need(stages);
  cudaError_t e;
  int per_sm = 0;
  for (void* kf : {tma_kernel<false>(TK), tma_kernel<true>(TK)})
    if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_kernel<false>(TK), threads, sm);
  if (e || per_sm < 1) {
    cudaGetLastError();
    return cudaSuccess;
  }
  c->tmy_stages = stages;
  c->tmy_tk = TK;
  c->tmy_threads = threads;
  c->tmy_smem = sm;
  c->tmy_blocks_per_sm = per_sm;
  c->tma_y = 1;
  return cudaSuccess;
}

template <typename R, int TK>
static void launch_tma(afid_ctx* c, const typename cplx<R>::T* tw, bool inv, const double* skip) {
  const Grid& g = c->g;
  const int ntile_x = ceil_div(g.M + 1, TK);
  const long long ntiles = (long long)ntile_x * g.nz;
  long long blocks = (long long)c->num_sms * c->tmy_blocks_per_sm;
  if (blocks > ntiles) blocks = ntiles;
  auto kf = inv ? k_fft_y_tma<R, true, TK> : k_fft_y_tma<R, false, TK>;
  // a stall requested by afid_test_tma_timeout applies to one launch, with a
  // 1 ms wait limit
  const int stall = c->tma_stall_once ? 0 : -1;
  const uint64_t limit = c->tma_stall_once ? 1000000ull : kWaitLimitNs;
  c->tma_stall_once = 0;
  kf<<<(int)blocks, c->tmy_threads, c->tmy_smem, c->stream>>>(c->tmy, g, tw, skip, c->scal, c->tmy_stages,
                                                               ntile_x, stall, limit);
}

template <typename R>
cudaError_t run_fft_y_tma(afid_ctx* c, const typename cplx<R>::T* tw, bool inv, const double* skip) {
  if (c->tmy_tk == 16) launch_tma<R, 16>(c, tw, inv, skip);
  else if (c->tmy_tk == 8) launch_tma<R, 8>(c, tw, inv, skip);
  else launch_tma<R, 4>(c, tw, inv, skip);
  c->launches++;
  return cudaGetLastError();
}

template cudaError_t run_fft_y_tma<float>(afid_ctx*, const float2*, bool, const double*);

}  // namespace afid

extern "C" afid_status afid_test_tma_timeout(afid_ctx* c) {
  if (!c) return AFID_ERR_INVALID_ARG;
  if (!c->tma_y) return AFID_ERR_INVALID_ARG;  // no TMA transform on this context
  c->tma_stall_once = 1;
  return AFID_OK;
}
