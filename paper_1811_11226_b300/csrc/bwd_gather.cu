// Input-driven adjoint of the image warp with respect to the input volume: a
// gather over the inverse footprint.
//
// grad_in[n] = a sum_o g(o) w_n(o), where output voxel o contributes to input
// voxel n exactly when n is one of the 8 taps of its cell, i.e. when
// floor(s_r(o)) is n_r - 1 or n_r on every axis r, i.e. s(o) = A o + b lies in
// the box [n - 1, n + 1).  Those o lie in the parallelepiped A^-1 (box - b),
// centred at c = A^-1 (n - b) with half-widths h_c = sum_r |A^-1_cr| along
// output axis c.  One thread per input voxel walks the output grid points of
// that bounding box (clipped to the output), decides membership and the
// weight from the exact Q.40 coordinate of each (the same cell and weight as
// the forward and the scatter adjoint: w_n = prod_r (n_r == floor(s_r) ?
// 1 - t_r : t_r)), and writes its sum with a plain store.  The box is found in
// float with a margin far above float rounding, so it never misses a
// contributing o; the exact test rejects the others.
//
// Each sum is taken by one thread in a fixed order, so grad_in is bitwise
// reproducible, needs no zeroing pass and no atomics.  The affine gradient is
// the output-driven pass of bwd.cuh (launch_bwd runs it after this kernel).
#include "bwd.cuh"

namespace augk {

// grad_in of input voxels (x, y, z0 .. z1 - 1) of one thread.  The box centre
// of (x, y, z0) is taken in double (the offset of the affine may be large) and
// clamped to a range beyond which no output point can lie in the box; the
// steps along z are float (at most a few tens of voxels).
__device__ __forceinline__ void gather_run(const VolConst& vc, int x, int y, int z0, int z1,
                                           bool valid, const float* __restrict__ g,
                                           float* gin) {
  const int onx = vc.onx, ony = vc.ony, onz = vc.onz;
  const long long ax = vc.tq[0][0], ay = vc.tq[1][0], az = vc.tq[2][0];
  const int klo = vc.occ_klo, khi = vc.occ_khi;
  const int nxy = vc.nx * vc.ny;
  const int on[3] = {onx, ony, onz};
  float oc0[3], dz[3], h[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double o = vc.ainv[c][0] * x + vc.ainv[c][1] * y + vc.ainv[c][2] * z0 + vc.binv[c];
    oc0[c] = (float)fmin(fmax(o, -32768.0), 32768.0);
    dz[c] = (float)vc.ainv[c][2];
    h[c] = vc.inv_h[c];
  }
  for (int z = z0; z < z1; ++z) {
    int lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float oc = fmaf(dz[c], (float)(z - z0), oc0[c]);
      lo[c] = max((int)ceilf(oc - h[c]), 0);
      hi[c] = min((int)floorf(oc + h[c]), on[c] - 1);
    }
    float acc = 0.0f;
    for (int k = lo[2]; k <= hi[2]; ++k) {
      if (k >= klo && k <= khi) continue;  // occluded outputs pass no gradient
      for (int j = lo[1]; j <= hi[1]; ++j) {
        long long sx = coord_q40(vc.tq[0], lo[0], j, k);
        long long sy = coord_q40(vc.tq[1], lo[0], j, k);
        long long sz = coord_q40(vc.tq[2], lo[0], j, k);
        const float* gr = g + ((size_t)k * ony + j) * onx;
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const int ex = x - q40_floor(sx), ey = y - q40_floor(sy), ez = z - q40_floor(sz);
          if ((unsigned)ex <= 1u && (unsigned)ey <= 1u && (unsigned)ez <= 1u) {
            const float tx = q40_frac(sx), ty = q40_frac(sy), tz = q40_frac(sz);
            const float wx = ex == 0 ? 1.0f - tx : tx;
            const float wy = ey == 0 ? 1.0f - ty : ty;
            const float wz = ez == 0 ? 1.0f - tz : tz;
            acc = fmaf(__ldg(gr + i), wx * wy * wz, acc);
          }
          sx += ax;
          sy += ay;
          sz += az;
        }
      }
    }
    if (valid) gin[(size_t)z * nxy + (size_t)y * vc.nx + x] = vc.a * acc;
  }
}

// Largest bounding box (output grid points per input voxel) the gather takes;
// beyond it (magnification of about 8x per axis, or a singular A) the volume
// is reported as unsupported.
constexpr float kMaxGatherBox = 4096.0f;

// Input tiles of 32 (x, lanes) x NW (y, warps) x ZT (z, per thread), static
// schedule over the concatenated input tile lists of all volumes.
template <int NW, int ZT>
__global__ void __launch_bounds__(NW * 32)
    k_bwd_gather(const aug_volume_desc* __restrict__ descs, int n_vols,
                 const VolConst* __restrict__ tab, const float* const* gout, float* const* gin,
                 WsHeader* ws) {
  __shared__ SchedSmem<NW * 32> sm;
  for_each_tile_t<NW, InBoxTiles<32, NW, ZT>>(
      descs, n_vols, sm, [&](int, int) {},
      [&](int v, int t, long long) {
        const VolConst& vc = tab[v];
        if (!vc.ok) return;
        const int ntx = (vc.nx + 31) / 32, nty = (vc.ny + NW - 1) / NW;
        const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
        const int x = tx * 32 + (int)(threadIdx.x & 31), y = ty * NW + (int)(threadIdx.x >> 5);
        const bool valid = x < vc.nx && y < vc.ny;
        const int z0 = tz * ZT, z1 = min(z0 + ZT, vc.nz);
        float* gi = gin[v];
        const float box = (2.0f * vc.inv_h[0] + 1.0f) * (2.0f * vc.inv_h[1] + 1.0f) *
                          (2.0f * vc.inv_h[2] + 1.0f);
        if (!vc.inv_ok || !(box <= kMaxGatherBox)) {
          // (Nearly) singular or strongly magnifying affine: reported, and
          // this volume's input gradient is zero.
          if (threadIdx.x == 0 && t == 0) record_error(ws, AUG_ERR_UNSUPPORTED, v);
          if (valid)
            for (int z = z0; z < z1; ++z)
              gi[(size_t)z * vc.nx * vc.ny + (size_t)y * vc.nx + x] = 0.0f;
          return;
        }
        gather_run(vc, min(x, vc.nx - 1), min(y, vc.ny - 1), z0, z1, valid, gout[v], gi);
      });
}

namespace {
using GatherK = void (*)(const aug_volume_desc*, int, const VolConst*, const float* const*,
                         float* const*, WsHeader*);
struct GatherVariant {
  int threads;
  GatherK k;
  const char* name;
};
const GatherVariant kGather[] = {
    {8 * 32, k_bwd_gather<8, 8>, "gather32x8x8"},
    {4 * 32, k_bwd_gather<4, 16>, "gather32x4x16"},
};
}  // namespace

int bwd_gather_num_variants() { return (int)(sizeof(kGather) / sizeof(kGather[0])); }
const char* bwd_gather_variant_name(int v) { return kGather[v].name; }

cudaError_t launch_bwd_gather(int variant, const aug_volume_desc* d, int n,
                              const float* const* gout, float* const* gin, VolConst* tab,
                              WsHeader* ws, cudaStream_t st) {
  const GatherVariant& gv = kGather[variant];
  const int grid = persistent_grid((const void*)gv.k, gv.threads, 0);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  gv.k<<<grid, gv.threads, 0, st>>>(d, n, tab, gout, gin, ws);
  return cudaGetLastError();
}

}  // namespace augk
