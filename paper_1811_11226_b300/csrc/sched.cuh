// Persistent tile scheduler shared by the batched kernels.
//
// The global work list is the concatenation, in batch order, of every
// volume's output tiles.  CTA b of a grid of G takes global tiles b, b+G,
// b+2G, ... (static round-robin, so CTAs running at the same time work on
// neighbouring tiles of the same volume and its input stays in L2).
//
// Volumes are processed in chunks of BLOCK (one volume per thread): each
// thread reads the output dimensions of one descriptor, and a block-wide scan
// turns the per-volume tile and voxel counts into prefix sums in shared
// memory.  The CTA then walks only its own tiles, so a volume in which it has
// no tile costs it nothing beyond that one parallel read.
#pragma once

#include "common.cuh"

namespace augk {

// Cap on the resident CTAs per SM of a persistent launch (grid = min(resident,
// cap) x SM count).
constexpr int kMaxCtasPerSm = 16;

template <int BLOCK>
struct SchedSmem {
  int tile_pre[BLOCK + 1];        // exclusive prefix of tiles within the chunk
  long long vox_pre[BLOCK + 1];   // exclusive prefix of output voxels within the chunk
  int warp_tiles[BLOCK / 32];
  long long warp_vox[BLOCK / 32];
};

// Output dims of a descriptor if they are valid, else 0 tiles / 0 voxels (the
// full descriptor check happens when the volume is staged).  FLAT: tiles of
// the flat plane mapping (tile_coord_flat), else 32 x NW x 4*QZ boxes.
template <int NW, int QZ, bool FLAT>
__device__ __forceinline__ void volume_counts(const aug_volume_desc* d, int& tiles,
                                              long long& vox) {
  const int onx = d->out_nx, ony = d->out_ny, onz = d->out_nz;
  const bool ok = onx >= 1 && ony >= 1 && onz >= 1 && onx <= MAX_DIM && ony <= MAX_DIM &&
                  onz <= MAX_DIM && (long long)onx * ony * onz < (1LL << 31);
  const int per_slab = FLAT ? (onx * ony + NW * 32 - 1) / (NW * 32)
                            : ((onx + 31) / 32) * ((ony + NW - 1) / NW);
  tiles = ok ? per_slab * ((onz + 4 * QZ - 1) / (4 * QZ)) : 0;
  vox = ok ? (long long)onx * ony * onz : 0;
}

// Calls body(v, local_tile, vox_offset) for every tile of this CTA, in
// increasing global order, with all threads of the CTA together (body may
// synchronise).  chunk_begin(c0, cnt) runs once per chunk before its tiles
// (all threads; may synchronise), e.g. to zero per-volume partial sums.
template <int NW, int QZ, bool FLAT = false, typename ChunkF, typename BodyF>
__device__ __forceinline__ void for_each_tile(const aug_volume_desc* __restrict__ descs,
                                              int n_vols, SchedSmem<NW * 32>& sm,
                                              ChunkF&& chunk_begin, BodyF&& body) {
  constexpr int BLOCK = NW * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long G = gridDim.x;
  long long gbase = 0;    // global index of the chunk's first tile
  long long voxbase = 0;  // output voxels before the chunk
  for (int c0 = 0; c0 < n_vols; c0 += BLOCK) {
    const int cnt = min(BLOCK, n_vols - c0);
    int t = 0;
    long long x = 0;
    if ((int)threadIdx.x < cnt) volume_counts<NW, QZ, FLAT>(descs + c0 + threadIdx.x, t, x);
    // Inclusive warp scan, then across warps.
    int ti = t;
    long long xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(FULL_MASK, ti, o);
      const long long b = __shfl_up_sync(FULL_MASK, xi, o);
      if (lane >= o) {
        ti += a;
        xi += b;
      }
    }
    __syncthreads();  // previous chunk's readers are done with sm
    if (lane == 31) {
      sm.warp_tiles[warp] = ti;
      sm.warp_vox[warp] = xi;
    }
    __syncthreads();
    int wt = 0;
    long long wx = 0;
    for (int w = 0; w < warp; ++w) {
      wt += sm.warp_tiles[w];
      wx += sm.warp_vox[w];
    }
    sm.tile_pre[threadIdx.x + 1] = wt + ti;
    sm.vox_pre[threadIdx.x + 1] = wx + xi;
    if (threadIdx.x == 0) {
      sm.tile_pre[0] = 0;
      sm.vox_pre[0] = 0;
    }
    __syncthreads();
    chunk_begin(c0, cnt);
    const int chunk_tiles = sm.tile_pre[cnt];
    int vi = 0;
    for (long long g = gbase + ((long long)blockIdx.x - gbase % G + G) % G;
         g < gbase + chunk_tiles; g += G) {
      const int lt = (int)(g - gbase);
      while (sm.tile_pre[vi + 1] <= lt) ++vi;
      body(c0 + vi, lt - sm.tile_pre[vi], voxbase + sm.vox_pre[vi]);
    }
    gbase += chunk_tiles;
    voxbase += sm.vox_pre[cnt];
  }
}

// Image requirement of a kernel's descriptors: never (IOU), when out_image is
// set (forward), always (adjoint).
enum { NEED_IMAGE_NEVER = 0, NEED_IMAGE_IF_OUT = 1, NEED_IMAGE_ALWAYS = 2 };

__device__ __forceinline__ bool needs_image(const aug_volume_desc& d, int need) {
  return need == NEED_IMAGE_ALWAYS || (need == NEED_IMAGE_IF_OUT && d.out_image != nullptr);
}

// Prologue of every batched call, one thread per volume: validates the
// descriptor (plus the per-op buffer pointers), records the first invalid one
// in the workspace status word, and writes the parsed per-volume constants
// (affine in Q.40, ok flag) to a table in the workspace.  The main kernels
// read a tile's constants straight from that table (L1-cached, no barrier).
__global__ void k_prepare(const aug_volume_desc* __restrict__ descs, int n_vols, int need,
                          int f32_only, const float* const* gout, float* const* gin,
                          int need_label, unsigned forbid_flags, VolConst* __restrict__ tab,
                          WsHeader* ws);

}  // namespace augk
