// de_noalloc.cu -- split-precision evaluation of caller rows without a handle
// and without any allocation (de_eval_noalloc in de.h).
//
// Every buffer the evaluation kernels need (run descriptor, state word, work
// list, |y| per row, the split copy of M and the A operand tiles) is carved
// out of one file-scope device array of kNoallocScratch bytes.  Its address
// is looked up once per device with cudaGetSymbolAddress.  The kernels that
// run are the ones de_eval uses for split precisions (k_prep_rows, k_fit_tc
// in evaluation mode), so the two entry points give identical results.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "de.h"
#include "de_internal.cuh"
#include "de_kernels.h"
#include "de_tcgen05.cuh"

namespace de {

constexpr size_t kNoallocScratch = (size_t)16 << 20;  // 16 MiB, fixed at build time
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratch];

// [0, 1024): descriptor and state word; then the work list, |y|, a zero
// shift (used when the caller passes none), the split copy of M, the A tiles.
constexpr size_t kNaStateOff = (sizeof(RunDesc) + 63) / 64 * 64;
static_assert(kNaStateOff + sizeof(RunState) <= 1024, "descriptor block overflows its 1 KiB slot");

struct NaLayout {
  size_t items, ynorm, shift, b, a, total;
};

static size_t na_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static NaLayout na_layout(size_t tiles, int dp, size_t b_bytes, size_t a_tile) {
  NaLayout L;
  L.items = 1024;
  L.ynorm = na_up(L.items + tiles * sizeof(int2), 256);
  L.shift = na_up(L.ynorm + tiles * kTileM * sizeof(float), 256);
  L.b = na_up(L.shift + (size_t)dp * sizeof(double), 1024);
  L.a = na_up(L.b + b_bytes, 1024);
  L.total = L.a + tiles * a_tile;
  return L;
}

// Descriptor, zeroed state word, work list (run 0, tile t) and, when the
// caller gave no shift, a zero shift.
__global__ void k_noalloc_setup(RunDesc R, RunDesc* desc, RunState* st, int2* items, int tiles, double* zshift,
                                int dp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (t == 0) {
    *desc = R;
    RunState z;
    memset(&z, 0, sizeof z);
    *st = z;
  }
  for (int k = t; k < tiles; k += stride) items[k] = make_int2(0, k);
  if (zshift)
    for (int j = t; j < dp; j += stride) zshift[j] = 0.0;
}

// Round-to-nearest-even float -> bf16 bits (Inf/NaN truncated).
__device__ __forceinline__ uint16_t na_bf16_rn(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
// Round half away from zero to the 10 mantissa bits of tf32.
__device__ __forceinline__ float na_tf32_rna(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

// Split copy of M (row n = output coordinate) in the B operand layout of the
// tensor-core kernel: N tiles of ntn rows, each a high and a low part in the
// canonical K-major layout with ntn / 8 row groups; every byte of the
// npad x kpad region is written (zero outside d x d).
template <int ESZ>
__global__ void k_noalloc_pack_b(const double* __restrict__ M, int d, int ntn, int kpad, int npad,
                                 uint8_t* __restrict__ B) {
  const size_t part = (size_t)ntn * kpad * ESZ;
  const int RG = ntn / 8, per = 16 / ESZ;
  const long long total = (long long)npad * kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / kpad), k = (int)(e % kpad);
    double mv = 0.0;
    if (n < d && k < d) mv = M ? M[(size_t)n * d + k] : (n == k ? 1.0 : 0.0);
    const float mf = __double2float_rn(mv);
    const int nt = n / ntn, nl = n % ntn;
    const size_t off = (size_t)nt * 2 * part + (((size_t)(k / per) * RG + nl / 8) * 128) + (nl % 8) * 16 +
                       (size_t)(k % per) * ESZ;
    if (ESZ == 2) {
      const uint16_t hi = na_bf16_rn(mf);
      const uint16_t lo = na_bf16_rn(__fsub_rn(mf, __uint_as_float((uint32_t)hi << 16)));
      *reinterpret_cast<uint16_t*>(B + off) = hi;
      *reinterpret_cast<uint16_t*>(B + off + part) = lo;
    } else {
      const float hi = na_tf32_rna(mf);
      const float lo = na_tf32_rna(__fsub_rn(mf, hi));
      *reinterpret_cast<float*>(B + off) = hi;
      *reinterpret_cast<float*>(B + off + part) = lo;
    }
  }
}

// Bytes one call needs for d (one 128-row tile), by the geometry rules below.
static size_t na_one_tile_bytes(int d, int esz) {
  const int kpad = (int)na_up(d, 16);
  const int ntn = d <= 256 ? kpad : 256;
  const int nn = (d + ntn - 1) / ntn;
  const size_t a_tile = (size_t)2 * kTileM * kpad * esz, b_tile = (size_t)2 * ntn * kpad * esz;
  return na_layout(1, (d + 3) / 4 * 4, nn * b_tile, a_tile).total;
}

// Largest d whose split copy of M and one operand tile fit the scratch
// (1920 for BF16X3, 1280 for TF32X3); the need grows with d.
static int na_max_d(int esz) {
  int d = 4096;
  while (d > 1 && na_one_tile_bytes(d, esz) > kNoallocScratch) --d;
  return d;
}

static std::mutex g_na_mu;
static uint8_t* g_na_base[kNoallocMaxDevices];

de_status noalloc_eval(int prec, int obj, int d, double scale, const double* o, const double* M, const double* x,
                       int64_t ld, int n, double* f, cudaStream_t s, std::string& err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoallocMaxDevices) {
    err = "de_eval_noalloc: device ordinal beyond " + std::to_string(kNoallocMaxDevices - 1);
    return DE_ERR_UNSUPPORTED;
  }
  uint8_t* base = nullptr;
  {
    // one-time set-up on this device: the scratch's device address
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_base[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        err = std::string("de_eval_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return DE_ERR_CUDA;
      }
      g_na_base[dev] = (uint8_t*)p;
    }
    base = g_na_base[dev];
  }

  // geometry of the tensor-core evaluation (the same rules as a handle's plan)
  const int esz = prec == DE_PREC_BF16X3 ? 2 : 4;
  const int kpad = (int)na_up(d, 16);
  const int ntn = d <= 256 ? kpad : 256;
  const int nn = (d + ntn - 1) / ntn;
  const int npad = nn * ntn;
  int kc;
  if ((size_t)2 * (kTileM + ntn) * kpad * esz <= kSingleStageMax) {
    kc = kpad;
  } else {
    kc = (int)(kStageBudget / (2 * (kTileM + ntn) * esz)) / 16 * 16;
    kc = std::max(16, std::min(kc, kpad));
  }
  const size_t stage = 2 * (size_t)(kc * esz / 16) * 16 * 128 + 2 * (size_t)(kc * esz / 16) * (ntn / 8) * 128;
  const size_t smem = (kc < kpad || nn > 1 ? 2 : 1) * stage;
  const size_t a_tile = (size_t)2 * kTileM * kpad * esz;
  const size_t b_tile = (size_t)2 * ntn * kpad * esz;
  const int dp = (d + 3) / 4 * 4;

  const size_t tiles = ((size_t)n + kTileM - 1) / kTileM;
  const NaLayout L = na_layout(tiles, dp, nn * b_tile, a_tile);
  if (na_layout(1, dp, nn * b_tile, a_tile).total > kNoallocScratch) {
    err = "de_eval_noalloc: d = " + std::to_string(d) + " does not fit the 16 MiB static scratch even for one " +
          "128-row tile; the largest d is " + std::to_string(na_max_d(esz)) + (esz == 2 ? " in BF16X3" : " in TF32X3");
    return DE_ERR_INVALID_ARG;
  }
  if (L.total > kNoallocScratch) {
    size_t tmax = std::min(tiles, kNoallocScratch / a_tile + 1);
    while (tmax > 0 && na_layout(tmax, dp, nn * b_tile, a_tile).total > kNoallocScratch) --tmax;
    err = "de_eval_noalloc: n = " + std::to_string(n) + " rows exceed the 16 MiB static scratch; for d = " +
          std::to_string(d) + (esz == 2 ? " in BF16X3" : " in TF32X3") + " at most " +
          std::to_string(tmax * kTileM) + " rows fit per call";
    return DE_ERR_INVALID_ARG;
  }

  RunDesc R;
  memset(&R, 0, sizeof R);
  R.np = n;
  R.d = d;
  R.dp = dp;
  R.obj = obj;
  R.scale = scale;
  R.unit_scale = scale == 1.0;
  R.rotate = M != nullptr;
  R.prec = prec;
  R.nw = (d + 31) / 32;
  R.o = o ? o : (const double*)(base + L.shift);
  R.st = (RunState*)(base + kNaStateOff);
  R.A = base + L.a;
  R.B = base + L.b;
  R.ynorm = (float*)(base + L.ynorm);
  R.kpad = kpad;
  R.npad = npad;
  R.ntiles_tc = (int)tiles;
  R.kc = kc;
  R.nstage = kc < kpad || nn > 1 ? 2 : 1;
  R.ntn = ntn;
  R.nn = nn;
  R.esz = esz;
  R.a_tile_bytes = (int)a_tile;
  R.b_tile_bytes = (int)b_tile;
  R.band_u = (float)((esz == 2 ? 3.0 * std::ldexp(1.0, -16) : 3.0 * std::ldexp(1.0, -22)) + kpad * std::ldexp(1.0, -24));

  RunDesc* desc = (RunDesc*)base;
  int2* items = (int2*)(base + L.items);
  k_noalloc_setup<<<1, 256, 0, s>>>(R, desc, R.st, items, (int)tiles, o ? nullptr : (double*)(base + L.shift), dp);
  const long long pack_n = (long long)npad * kpad;
  const int pack_grid = (int)std::min<long long>((pack_n + 255) / 256, 1024);
  if (esz == 2)
    k_noalloc_pack_b<2><<<pack_grid, 256, 0, s>>>(M, d, ntn, kpad, npad, base + L.b);
  else
    k_noalloc_pack_b<4><<<pack_grid, 256, 0, s>>>(M, d, ntn, kpad, npad, base + L.b);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("de_eval_noalloc: set-up launch: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  return tc_eval_rows(desc, items, (int)tiles, esz, smem, x, ld, n, f, s, err);
}

}  // namespace de
