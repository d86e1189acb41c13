// Anti-aliasing Gaussian of the resampling step (Sec. 5.A):
//   S(p) = sum_{a,b,c} wx[a] wy[b] wz[c] E(p + (a, b, c)),
// wk the normalised 1-D weights of exp(-x^2 / sigma_k^2) on |x| <= ceil(3 sigma_k),
// E the input extended by the fill value.  The filter is separable; one pass
// over the volume does all three axes:
//
//   * a CTA owns a column of 64 (x) x 16 (y) outputs over a z-chunk of 128
//     slices and walks the input slices of that chunk plus R on either side;
//   * each input slice tile (16 + 2R rows) arrives in shared memory by a TMA
//     tensor copy issued two slices ahead into a double buffer (an mbarrier
//     per buffer), so no thread spends instructions or waits on its loads;
//     volumes whose row pitch is not a multiple of 16 bytes are staged by
//     per-thread loads instead;
//   * the tile is converted to float (int16 by an exact integer trick) with
//     the fill value patched in outside the volume, then the x pass (two
//     adjacent outputs per thread and row) and the y pass (two adjacent rows of
//     two outputs per thread, packed f32x2 FMAs) run on it;
//   * the y-filtered pairs of the last 2R + 1 slices stay in registers (a ring
//     with compile-time indices: the slice loop is unrolled by 2R + 1), and the
//     z pass combines them into the output slice R behind the newest one.
//
// DRAM traffic is one read of the input (halo re-reads hit L2) and one float32
// write per voxel.  Volumes are launched in groups that share the input type,
// the padded radius R, the staging path and sigma, at most 32 per launch, by
// value.
//
// Every wait on an mbarrier is bounded; a CTA that gives up records status 1
// in the library's smoothing status word, waits (bounded) for its other copy
// in flight and returns.  Each TMA destination is a 128-byte aligned buffer.
#include <cuda.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "kernels.h"

namespace augk {

constexpr int kSmTX = 64;       // outputs along x per CTA
constexpr int kSmTY = 16;       // outputs along y per CTA (two rows per warp)
constexpr int kSmZC = 128;      // output slices per CTA
constexpr int kSmMaxR = 8;      // largest supported radius
constexpr int kSmMaxVols = 32;  // volumes per launch
constexpr int kSmBoxX = kSmTX + 16;  // TMA box: columns tx0 - 8 .. tx0 + 71 (16-byte aligned start)

struct SmoothVol {
  CUtensorMap tmap;  // used by the TMA path only
  const void* in;
  float* out;
  int nx, ny, nz;
  int tiles_x, tiles_xy;  // tiles along x, x*y
  int vec_store;          // nx even and out 8-byte aligned: paired stores
  float fill;
};

// One launch: volumes with the same input type, radius, staging path and
// sigma, so that the weights sit at fixed parameter offsets (the FMAs read
// them from the constant bank instead of registers).
struct SmoothBatch {
  // First, so that it lies in the first 4 KB of the parameters, where
  // instructions can read it directly.
  float w[3][2 * kSmMaxR + 1];  // per axis, offset a at [kSmMaxR + a]; zero outside its radius
  int n;
  int no_copies;  // test of the bounded waits: issue no tile copy, so every wait runs out
  int* status;
  int tile_start[kSmMaxVols + 1];  // exclusive prefix of CTA tiles
  SmoothVol v[kSmMaxVols];
};

__device__ int g_smooth_status;

// ---- small PTX helpers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with the given parity (about a second at most).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it >= 16) __nanosleep(64);
  }
  return false;
}
// 3-D tiled TMA load of box (x, y, z) of `map` into shared memory.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// int16 -> float without the conversion unit: 0x4B400000 is 1.5 * 2^23, so
// its bit pattern plus v (|v| < 2^22) is the float 1.5 * 2^23 + v exactly.
__device__ __forceinline__ float i16_to_f(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

template <typename TIn>
__device__ __forceinline__ float ld_global(const TIn* p);
template <>
__device__ __forceinline__ float ld_global<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ld_global<int16_t>(const int16_t* p) {
  return i16_to_f(__ldg(p));
}

// Compile-time shape of a CTA's staged tile for radius R.
template <typename TIn, int R>
struct SmTile {
  static constexpr int W = kSmTX + 2 * R;  // staged columns
  static constexpr int H = kSmTY + 2 * R;  // staged rows
  static constexpr int K = 2 * R + 1;      // taps per axis
  static constexpr int PAIRS = H * (W / 2);
  static constexpr uint32_t BOX_BYTES = (uint32_t)(kSmBoxX * H * sizeof(TIn));
  // A tiled TMA copy needs a 128-byte aligned shared destination: each
  // buffer starts on a 128-byte boundary.
  static constexpr uint32_t RAW_STRIDE = (BOX_BYTES + 127u) / 128u * 128u;
};

// in_t (float, H x W) <- the TMA box raw (H x kSmBoxX, columns from tx0 - 8).
// PATCH: put the fill value where the tile lies outside the volume.
template <typename TIn, int R, bool PATCH>
__device__ __forceinline__ void convert_raw(const TIn* raw, float* in_t, int tx0, int ty0, int nx,
                                            int ny, float fill) {
  using T = SmTile<TIn, R>;
#pragma unroll
  for (int i = 0; i < (T::PAIRS + 255) / 256; ++i) {
    const int e = (int)threadIdx.x + 256 * i;
    if (e < T::PAIRS) {
      const int r = e / (T::W / 2), c = 2 * (e - r * (T::W / 2));
      const TIn* src = raw + r * kSmBoxX + c + 8 - R;
      float v0, v1;
      if (sizeof(TIn) == 2) {
        if ((8 - R) % 2 == 0) {
          // two int16 in one aligned 32-bit word (little-endian)
          const int wrd = *reinterpret_cast<const int*>(src);
          v0 = i16_to_f((int)((unsigned)wrd << 16) >> 16);
          v1 = i16_to_f(wrd >> 16);
        } else {
          const int16_t* s16 = reinterpret_cast<const int16_t*>(src);
          v0 = i16_to_f(s16[0]);
          v1 = i16_to_f(s16[1]);
        }
      } else {
        const float* s32 = reinterpret_cast<const float*>(src);
        v0 = s32[0];
        v1 = s32[1];
      }
      if (PATCH) {
        const int gx = tx0 - R + c, gy = ty0 - R + r;
        const bool y_in = gy >= 0 && gy < ny;
        if (!(y_in && gx >= 0 && gx < nx)) v0 = fill;
        if (!(y_in && gx + 1 < nx && gx + 1 >= 0)) v1 = fill;
      }
      *reinterpret_cast<float2*>(in_t + r * T::W + c) = make_float2(v0, v1);
    }
  }
}

// in_t <- slice zi of the volume by per-thread loads (volumes without a TMA map).
template <typename TIn, int R, bool PATCH>
__device__ __forceinline__ void load_direct(const TIn* slice, float* in_t, int tx0, int ty0,
                                            int nx, int ny, float fill) {
  using T = SmTile<TIn, R>;
#pragma unroll
  for (int i = 0; i < (T::H * T::W + 255) / 256; ++i) {
    const int e = (int)threadIdx.x + 256 * i;
    if (e < T::H * T::W) {
      const int r = e / T::W, c = e - r * T::W;
      const int gx = tx0 - R + c, gy = ty0 - R + r;
      if (PATCH)
        in_t[e] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx)
                      ? ld_global<TIn>(slice + (size_t)gy * nx + gx)
                      : fill;
      else
        in_t[e] = ld_global<TIn>(slice + (size_t)gy * nx + gx);
    }
  }
}

template <int... Us, typename F>
__device__ __forceinline__ bool for_each_slot(std::integer_sequence<int, Us...>, F&& f) {
  return (f(std::integral_constant<int, Us>{}) && ...);
}

template <typename TIn, int R, bool TMA>
__global__ void __launch_bounds__(256, R <= 4 ? 3 : 2)
    k_smooth(const __grid_constant__ SmoothBatch B) {
  using T = SmTile<TIn, R>;
  constexpr int W = T::W, H = T::H, K = T::K;
  constexpr uint32_t RAW_STRIDE = TMA ? T::RAW_STRIDE : 128u;
  static_assert(RAW_STRIDE % 128u == 0u, "TMA buffers must be 128-byte aligned");
  __shared__ __align__(128) unsigned char raw_bytes[2 * RAW_STRIDE];
  __shared__ __align__(16) float in_t[H * W];
  __shared__ __align__(16) float xt[H][kSmTX];
  __shared__ __align__(8) unsigned long long bar[2];

  // Volume and tile of this CTA (uniform scan over at most 32 entries).
  int vi = 0;
  while (vi + 1 < B.n && (int)blockIdx.x >= B.tile_start[vi + 1]) ++vi;
  const SmoothVol& V = B.v[vi];
  const int t = (int)blockIdx.x - B.tile_start[vi];
  const int tz = t / V.tiles_xy, txy = t - tz * V.tiles_xy;
  const int ty0 = (txy / V.tiles_x) * kSmTY, tx0 = (txy % V.tiles_x) * kSmTX;
  const int z0 = tz * kSmZC, z1 = min(z0 + kSmZC, V.nz);
  const int nx = V.nx, ny = V.ny, nz = V.nz;
  const float fill = V.fill;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int px = 2 * lane;  // first of two x outputs of this thread
  // Weights: B.w at fixed offsets (tap a of axis k is B.w[k][kSmMaxR - R + a]);
  // the x pass reads them from the parameter bank, the y and z passes use
  // register pairs (w, w) for the packed FMAs.
  const float(&wt)[3][2 * kSmMaxR + 1] = B.w;
  f32x2 wy2[K], wz2[K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    wy2[a] = pk2(wt[1][kSmMaxR - R + a], wt[1][kSmMaxR - R + a]);
    wz2[a] = pk2(wt[2][kSmMaxR - R + a], wt[2][kSmMaxR - R + a]);
  }
  const bool interior_xy =
      tx0 - R >= 0 && tx0 + W - R <= nx && ty0 - R >= 0 && ty0 + H - R <= ny;
  const int ox = tx0 + px;
  const bool pair_ok = ox + 1 < nx;
  const bool vec_store = V.vec_store != 0;

  const int zs = z0 - R, ze = z1 + R;  // input slices of this CTA
  uint32_t phase = 0;                  // bit b: parity of buffer b's next phase
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(smem_u32(&bar[0]), 1);
      mbar_init(smem_u32(&bar[1]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // Guard: never issue a copy to a misaligned destination (cannot happen by
    // construction; recorded as an error and the CTA leaves).
    if ((smem_u32(raw_bytes) & 127u) != 0u) {
      if (threadIdx.x == 0) atomicExch(B.status, 2);
      return;
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < 2; ++i) {
        const int zi = zs + i;
        if (zi < ze && zi >= 0 && zi < nz && !B.no_copies) {
          mbar_expect_tx(smem_u32(&bar[i]), T::BOX_BYTES);
          tma_load_3d(smem_u32(raw_bytes + i * RAW_STRIDE), &V.tmap, tx0 - 8, ty0 - R, zi,
                      smem_u32(&bar[i]));
        }
      }
    }
  }

  f32x2 ring0[K], ring1[K];  // output rows 2 warp and 2 warp + 1
#pragma unroll
  for (int c = 0; c < K; ++c) ring0[c] = ring1[c] = pk2(0.0f, 0.0f);

  // One input slice; U (compile time) is its ring slot, zi = zb + U.  OUT: the
  // slice completes an output slice (every slice but the first 2R of the CTA);
  // FULL: every output of the tile lies inside the volume.  Returns false when
  // the CTA must stop (a copy never arrived).
  int zb = zs;
  const bool full_tile = tx0 + kSmTX <= nx && ty0 + kSmTY <= ny;
  auto step = [&](auto slot, auto out_c, auto full_c) -> bool {
    constexpr int U = decltype(slot)::value;
    constexpr bool OUT = decltype(out_c)::value;
    constexpr bool FULL = decltype(full_c)::value;
    const int zi = zb + U;
    if (zi >= ze) return true;
    const int b = (zi - zs) & 1;
    const bool z_in = zi >= 0 && zi < nz;
    // ---- stage the slice tile as float in in_t ----------------------------------------
    bool ok = true;
    if (!z_in) {
      for (int e = threadIdx.x; e < H * W; e += 256) in_t[e] = fill;
    } else if (TMA) {
      ok = mbar_wait(smem_u32(&bar[b]), (phase >> b) & 1u);
      phase ^= 1u << b;
      const TIn* raw = reinterpret_cast<const TIn*>(raw_bytes + b * RAW_STRIDE);
      if (interior_xy)
        convert_raw<TIn, R, false>(raw, in_t, tx0, ty0, nx, ny, fill);
      else
        convert_raw<TIn, R, true>(raw, in_t, tx0, ty0, nx, ny, fill);
    } else {
      const TIn* slice = (const TIn*)V.in + (size_t)zi * (size_t)nx * (size_t)ny;
      if (interior_xy)
        load_direct<TIn, R, false>(slice, in_t, tx0, ty0, nx, ny, fill);
      else
        load_direct<TIn, R, true>(slice, in_t, tx0, ty0, nx, ny, fill);
    }
    if (__syncthreads_or(!ok)) {
      // A copy never arrived: record it, wait once more (bounded) for the
      // copies that may still be in flight (this slice's and the next one's),
      // and leave.
      if (threadIdx.x == 0) {
        atomicExch(B.status, 1);
        if (TMA) {
          if (!B.no_copies) mbar_wait(smem_u32(&bar[b]), ((phase >> b) & 1u) ^ 1u);
          const int zn = zi + 1;
          if (zn < ze && zn >= 0 && zn < nz && !B.no_copies)
            mbar_wait(smem_u32(&bar[b ^ 1]), (phase >> (b ^ 1)) & 1u);
        }
      }
      return false;
    }
    // raw[b] is consumed: fetch the slice two ahead into it.
    if (TMA && threadIdx.x == 0) {
      const int zn = zi + 2;
      if (zn < ze && zn >= 0 && zn < nz && !B.no_copies) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(smem_u32(&bar[b]), T::BOX_BYTES);
        tma_load_3d(smem_u32(raw_bytes + b * RAW_STRIDE), &V.tmap, tx0 - 8, ty0 - R, zn,
                    smem_u32(&bar[b]));
      }
    }
    // ---- x pass: rows warp, warp + 8, ..., two outputs each ----------------------------
#pragma unroll
    for (int m = 0; m < (H + 7) / 8; ++m) {
      const int r = warp + 8 * m;
      if (r < H) {
        const float2* src = reinterpret_cast<const float2*>(in_t + r * W + px);
        float v[K + 1];
#pragma unroll
        for (int j = 0; j < (K + 1) / 2; ++j) {
          const float2 q = src[j];
          v[2 * j] = q.x;
          v[2 * j + 1] = q.y;
        }
        float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const float w = wt[0][kSmMaxR - R + a];
          a0 = fmaf(w, v[a], a0);
          a1 = fmaf(w, v[a + 1], a1);
        }
        *reinterpret_cast<float2*>(&xt[r][px]) = make_float2(a0, a1);
      }
    }
    __syncthreads();
    // ---- y pass: output rows 2 warp and 2 warp + 1 (rows 2 warp .. 2 warp + 2R + 1 of xt)
    f32x2 y0 = pk2(0.0f, 0.0f), y1 = pk2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k <= K; ++k) {
      const float2 q = *reinterpret_cast<const float2*>(&xt[2 * warp + k][px]);
      if (k < K) y0 = fma2(wy2[k], pk2(q.x, q.y), y0);
      if (k > 0) y1 = fma2(wy2[k - 1], pk2(q.x, q.y), y1);
    }
    // ---- z pass: slot U holds slice zb + U; slice zo - R + c is in slot (U + 1 + c) mod K
    ring0[U] = y0;
    ring1[U] = y1;
    const int zo = zi - R;
    if (OUT && (FULL || ox < nx)) {
      f32x2 o0 = pk2(0.0f, 0.0f), o1 = pk2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < K; ++c) {
        o0 = fma2(wz2[c], ring0[(U + 1 + c) % K], o0);
        o1 = fma2(wz2[c], ring1[(U + 1 + c) % K], o1);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int oy = ty0 + 2 * warp + h;
        if (FULL || oy < ny) {
          float a, c;
          upk2(h == 0 ? o0 : o1, a, c);
          float* dst = V.out + ((size_t)zo * ny + oy) * (size_t)nx + ox;
          if ((FULL || pair_ok) && vec_store) {
            __stcs(reinterpret_cast<float2*>(dst), make_float2(a, c));
          } else {
            __stcs(dst, a);
            if (pair_ok) __stcs(dst + 1, c);
          }
        }
      }
    }
    return true;
  };
  // The first round holds the CTA's first K input slices: only its last slot
  // completes an output slice.  Later rounds complete one per slot.
  auto run = [&](auto full_c) -> bool {
    if (!for_each_slot(std::make_integer_sequence<int, K>{}, [&](auto slot) {
          constexpr int U = decltype(slot)::value;
          return step(slot, std::integral_constant<bool, U == K - 1>{}, full_c);
        }))
      return false;
#pragma unroll 1
    for (zb += K; zb < ze; zb += K)
      if (!for_each_slot(std::make_integer_sequence<int, K>{}, [&](auto slot) {
            return step(slot, std::true_type{}, full_c);
          }))
        return false;
    return true;
  };
  if (full_tile)
    run(std::true_type{});
  else
    run(std::false_type{});
}

namespace {

using SmoothK = void (*)(const SmoothBatch);

template <int R>
SmoothK smooth_kernel(int dtype, bool tma) {
  if (dtype == AUG_I16)
    return tma ? (SmoothK)k_smooth<int16_t, R, true> : (SmoothK)k_smooth<int16_t, R, false>;
  return tma ? (SmoothK)k_smooth<float, R, true> : (SmoothK)k_smooth<float, R, false>;
}

SmoothK pick(int dtype, int R, bool tma) {
  switch (R) {
    case 1: return smooth_kernel<1>(dtype, tma);
    case 2: return smooth_kernel<2>(dtype, tma);
    case 3: return smooth_kernel<3>(dtype, tma);
    case 4: return smooth_kernel<4>(dtype, tma);
    case 6: return smooth_kernel<6>(dtype, tma);
    default: return smooth_kernel<8>(dtype, tma);
  }
}

int padded_radius(int r) {
  if (r <= 1) return 1;
  if (r <= 4) return r;
  return r <= 6 ? 6 : 8;
}

// cuTensorMapEncodeTiled, fetched from the driver through the runtime (no
// link-time dependency on the driver library).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  });
  return fn;
}

// TMA tensor map of a volume, box (kSmBoxX, 16 + 2R, 1); false when the
// volume's layout does not allow one (row pitch or base not 16-byte aligned).
bool make_tmap(const aug_smooth_desc& d, int R, CUtensorMap* m) {
  const size_t e = d.image_dtype == AUG_I16 ? 2 : 4;
  if (((size_t)d.nx * e) % 16 != 0 || (uintptr_t)d.image % 16 != 0) return false;
  EncodeTiled enc = encode_fn();
  if (enc == nullptr) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)d.nx * e, (cuuint64_t)d.nx * d.ny * e};
  const cuuint32_t box[3] = {(cuuint32_t)kSmBoxX, (cuuint32_t)(kSmTY + 2 * R), 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(m, e == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
             const_cast<void*>(d.image), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

int gauss_radius(float sigma) { return sigma > 0.0f ? (int)ceil(3.0 * (double)sigma) : 0; }

// Normalised weights of exp(-a^2 / sigma^2), |a| <= ceil(3 sigma), computed in
// double and rounded to float; w[kSmMaxR + a] for offset a, zero elsewhere.
static void gauss_weights(float sigma, float* w) {
  const int R = gauss_radius(sigma);
  double e[2 * kSmMaxR + 1], s = 0.0;
  for (int a = -R; a <= R; ++a) {
    e[R + a] = R == 0 ? 1.0 : exp(-(double)a * (double)a / ((double)sigma * (double)sigma));
    s += e[R + a];
  }
  for (int i = 0; i < 2 * kSmMaxR + 1; ++i) w[i] = 0.0f;
  for (int a = -R; a <= R; ++a) w[kSmMaxR + a] = (float)(e[R + a] / s);
}

int smooth_max_radius() { return kSmMaxR; }

cudaError_t smooth_status_word(int** p) {
  return cudaGetSymbolAddress((void**)p, g_smooth_status);
}

cudaError_t launch_smooth(const aug_smooth_desc* h, int n, cudaStream_t st, bool no_copies) {
  int* status = nullptr;
  cudaError_t e = smooth_status_word(&status);
  if (e != cudaSuccess) return e;
  // Per volume: padded radius and staging path; then groups of equal
  // (type, radius, path, sigma) in launches of <= 32 volumes.
  std::vector<int> rad(n);
  std::vector<char> tma(n);
  std::vector<CUtensorMap> maps(n);
  for (int b = 0; b < n; ++b) {
    const int r = std::max(gauss_radius(h[b].sigma[0]),
                           std::max(gauss_radius(h[b].sigma[1]), gauss_radius(h[b].sigma[2])));
    rad[b] = padded_radius(r);
    tma[b] = make_tmap(h[b], rad[b], &maps[b]);
  }
  // Groups of volumes with equal (type, radius, path, sigma), in first-seen order.
  std::vector<char> done(n, 0);
  std::vector<int> order;
  for (int b0 = 0; b0 < n; ++b0) {
    if (done[b0]) continue;
    order.clear();
    for (int b = b0; b < n; ++b)
      if (!done[b] && h[b].image_dtype == h[b0].image_dtype && rad[b] == rad[b0] &&
          tma[b] == tma[b0] && h[b].sigma[0] == h[b0].sigma[0] &&
          h[b].sigma[1] == h[b0].sigma[1] && h[b].sigma[2] == h[b0].sigma[2]) {
        order.push_back(b);
        done[b] = 1;
      }
    const int dtype = h[b0].image_dtype, R = rad[b0], path = tma[b0];
    for (size_t g0 = 0; g0 < order.size(); g0 += kSmMaxVols) {
      SmoothBatch* Bt = new SmoothBatch;  // ~12 KB: off the host stack
      Bt->n = 0;
      Bt->no_copies = no_copies ? 1 : 0;
      Bt->status = status;
      Bt->tile_start[0] = 0;
      for (int r = 0; r < 3; ++r) gauss_weights(h[b0].sigma[r], Bt->w[r]);
      for (size_t g = g0; g < order.size() && g < g0 + kSmMaxVols; ++g) {
        const aug_smooth_desc& d = h[order[g]];
        SmoothVol& V = Bt->v[Bt->n];
        V.tmap = maps[order[g]];
        V.in = d.image;
        V.out = d.out;
        V.nx = d.nx;
        V.ny = d.ny;
        V.nz = d.nz;
        V.tiles_x = (d.nx + kSmTX - 1) / kSmTX;
        V.tiles_xy = V.tiles_x * ((d.ny + kSmTY - 1) / kSmTY);
        V.vec_store = (d.nx % 2 == 0) && ((uintptr_t)d.out % 8 == 0);
        V.fill = d.fill;
        const long long tiles = (long long)V.tiles_xy * ((d.nz + kSmZC - 1) / kSmZC);
        if ((long long)Bt->tile_start[Bt->n] + tiles > 0x7fffffffLL) {
          delete Bt;
          return cudaErrorInvalidConfiguration;
        }
        Bt->tile_start[Bt->n + 1] = Bt->tile_start[Bt->n] + (int)tiles;
        ++Bt->n;
      }
      for (int i = Bt->n + 1; i <= kSmMaxVols; ++i) Bt->tile_start[i] = Bt->tile_start[Bt->n];
      pick(dtype, R, path != 0)<<<Bt->tile_start[Bt->n], 256, 0, st>>>(*Bt);
      e = cudaGetLastError();
      delete Bt;
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace augk
