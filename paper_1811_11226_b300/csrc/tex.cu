// The hardware-texture alternative to the forward warp: the paper's own way of
// sampling (Sec. 4, trilinear interpolation by the texture unit), measured
// beside the exact path.  Each float32 volume is copied once into a 3-D CUDA
// array read through a texture object with linear filtering and border
// addressing, the border colour being the fill value (so taps outside the
// volume read the fill, as in the exact path).  The coordinate is computed in
// float32 and the texture unit interpolates with its low-precision fixed-point
// weights; labels are the nearest voxel, read with an explicit bounds check.
// The intensity affine and the noise are those of the exact path (the same
// Philox stream), so the outputs differ only by the sampling.
//
// One launch per volume; a thread walks four z-consecutive voxels (one Philox
// call).  Float32 volumes only: a filtered integer texture returns normalised
// values, which would add its own error.
#include <vector>

#include "kernels.h"

namespace augk {
namespace {

struct TexVol {
  cudaTextureObject_t img;
  const uint8_t* lab;
  float* out_image;
  uint8_t* out_label;
  int nx, ny, nz, onx, ony, onz, fill_label;
  float T[12];
  float a, b, sigma;
  unsigned noise_id;
};

struct TexEntry {
  cudaArray_t arr = nullptr;
  cudaTextureObject_t tex = 0;
  aug_volume_desc d;
};

struct TexSet {
  std::vector<TexEntry> v;
};

constexpr int kTexNW = 4;

__global__ void __launch_bounds__(kTexNW * 32)
    k_tex_fwd(const TexVol V, const PhiloxKey key) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = blockIdx.y * kTexNW + (threadIdx.x >> 5);
  const int kq = blockIdx.z * 4;
  if (i >= V.onx || j >= V.ony) return;
  float z[4] = {0.f, 0.f, 0.f, 0.f};
  if (V.out_image && V.sigma > 0.0f) {
    const unsigned long long quad =
        ((unsigned long long)(kq >> 2) * (unsigned)V.ony + (unsigned)j) * (unsigned)V.onx +
        (unsigned)i;
    quad_normals(quad, V.noise_id, key, z);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int k = kq + m;
    if (k >= V.onz) break;
    const float fi = (float)i, fj = (float)j, fk = (float)k;
    const float sx = fmaf(V.T[0], fi, fmaf(V.T[1], fj, fmaf(V.T[2], fk, V.T[3])));
    const float sy = fmaf(V.T[4], fi, fmaf(V.T[5], fj, fmaf(V.T[6], fk, V.T[7])));
    const float sz = fmaf(V.T[8], fi, fmaf(V.T[9], fj, fmaf(V.T[10], fk, V.T[11])));
    const size_t o = ((size_t)k * V.ony + j) * V.onx + i;
    if (V.out_image) {
      // Texel centres sit at integer + 0.5 in unnormalised texture coordinates.
      const float v = tex3D<float>(V.img, sx + 0.5f, sy + 0.5f, sz + 0.5f);
      __stcs(V.out_image + o, fmaf(V.sigma, z[m], fmaf(V.a, v, V.b)));
    }
    if (V.out_label) {
      const int rx = (int)floorf(sx + 0.5f), ry = (int)floorf(sy + 0.5f),
                rz = (int)floorf(sz + 0.5f);
      int lab = V.fill_label;
      if ((unsigned)rx < (unsigned)V.nx && (unsigned)ry < (unsigned)V.ny &&
          (unsigned)rz < (unsigned)V.nz)
        lab = __ldg(V.lab + ((size_t)rz * V.ny + ry) * V.nx + rx);
      V.out_label[o] = (uint8_t)lab;
    }
  }
}

void destroy(TexSet* S) {
  for (TexEntry& e : S->v) {
    if (e.tex) cudaDestroyTextureObject(e.tex);
    if (e.arr) cudaFreeArray(e.arr);
  }
  delete S;
}

}  // namespace

aug_status tex_create(const aug_volume_desc* h, int n, void** handle) {
  TexSet* S = new TexSet;
  S->v.resize(n);
  for (int b = 0; b < n; ++b) {
    TexEntry& e = S->v[b];
    e.d = h[b];
    if (h[b].out_image == nullptr) continue;
    const cudaChannelFormatDesc cf = cudaCreateChannelDesc<float>();
    const cudaExtent ext = make_cudaExtent(h[b].in_nx, h[b].in_ny, h[b].in_nz);
    if (cudaMalloc3DArray(&e.arr, &cf, ext) != cudaSuccess) {
      destroy(S);
      return AUG_ERR_CUDA;
    }
    cudaMemcpy3DParms cp = {};
    cp.srcPtr = make_cudaPitchedPtr(const_cast<void*>(h[b].image), (size_t)h[b].in_nx * 4,
                                    h[b].in_nx, h[b].in_ny);
    cp.dstArray = e.arr;
    cp.extent = ext;
    cp.kind = cudaMemcpyDeviceToDevice;
    if (cudaMemcpy3D(&cp) != cudaSuccess) {
      destroy(S);
      return AUG_ERR_CUDA;
    }
    cudaResourceDesc rd = {};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = e.arr;
    cudaTextureDesc td = {};
    for (int r = 0; r < 3; ++r) td.addressMode[r] = cudaAddressModeBorder;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    td.borderColor[0] = h[b].fill_image;
    if (cudaCreateTextureObject(&e.tex, &rd, &td, nullptr) != cudaSuccess) {
      destroy(S);
      return AUG_ERR_CUDA;
    }
  }
  *handle = S;
  return AUG_OK;
}

aug_status tex_warp_fwd(void* handle, uint64_t seed, cudaStream_t st) {
  TexSet* S = (TexSet*)handle;
  const PhiloxKey key = philox_schedule((unsigned)seed, (unsigned)(seed >> 32));
  for (const TexEntry& e : S->v) {
    const aug_volume_desc& d = e.d;
    if (d.out_image == nullptr && d.out_label == nullptr) continue;
    TexVol V;
    V.img = e.tex;
    V.lab = d.label;
    V.out_image = e.tex ? d.out_image : nullptr;
    V.out_label = d.out_label;
    V.nx = d.in_nx;
    V.ny = d.in_ny;
    V.nz = d.in_nz;
    V.onx = d.out_nx;
    V.ony = d.out_ny;
    V.onz = d.out_nz;
    V.fill_label = d.fill_label;
    for (int m = 0; m < 12; ++m) V.T[m] = d.affine[m];
    V.a = d.photo_a;
    V.b = d.photo_b;
    V.sigma = d.noise_sigma;
    V.noise_id = d.noise_id;
    const dim3 grid((d.out_nx + 31) / 32, (d.out_ny + kTexNW - 1) / kTexNW, (d.out_nz + 3) / 4);
    k_tex_fwd<<<grid, kTexNW * 32, 0, st>>>(V, key);
    if (cudaGetLastError() != cudaSuccess) return AUG_ERR_CUDA;
  }
  return AUG_OK;
}

aug_status tex_destroy(void* handle) {
  if (handle) destroy((TexSet*)handle);
  return AUG_OK;
}

}  // namespace augk
