// Persistent tile scheduler shared by the batched kernels.
//
// The global work list is the concatenation, in batch order, of every
// volume's output tiles.  In the static form the CTAs take the tiles of each
// chunk of volumes round-robin (for_each_tile_t), so CTAs
// running at the same time work on neighbouring tiles of the same volume and
// its input stays in L2; in the dynamic form a CTA takes the next unclaimed
// tile of that list.
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
  long long next;                 // dynamic schedule: the CTA's current global tile
};

// Tile shapes of the schedulers: tiles(onx, ony, onz) per volume.
//  StdTiles<NW, QZ, FLAT>: the flat plane mapping (tile_coord_flat) when FLAT,
//    else boxes of 32 x NW x 4*QZ (tile_coord).
//  BoxTiles<TX, TY, TZ>: boxes of TX x TY x TZ, x fastest, then y, then z.
template <int NW, int QZ, bool FLAT>
struct StdTiles {
  __device__ __forceinline__ static int tiles(int onx, int ony, int onz) {
    const int per_slab = FLAT ? (onx * ony + NW * 32 - 1) / (NW * 32)
                              : ((onx + 31) / 32) * ((ony + NW - 1) / NW);
    return per_slab * ((onz + 4 * QZ - 1) / (4 * QZ));
  }
};
template <int TX, int TY, int TZ>
struct BoxTiles {
  __device__ __forceinline__ static int tiles(int onx, int ony, int onz) {
    return ((onx + TX - 1) / TX) * ((ony + TY - 1) / TY) * ((onz + TZ - 1) / TZ);
  }
};
// Boxes of TX x TY x TZ over the INPUT grid of each volume (input-driven
// kernels); counts input voxels.
template <int TX, int TY, int TZ>
struct InBoxTiles : BoxTiles<TX, TY, TZ> {
  static constexpr bool kInput = true;
};
template <typename T, typename = void>
struct tiles_over_input {
  static constexpr bool value = false;
};
template <typename T>
struct tiles_over_input<T, decltype((void)T::kInput)> {
  static constexpr bool value = T::kInput;
};

// Output dims of a descriptor if they are valid, else 0 tiles / 0 voxels (the
// full descriptor check happens when the volume is staged).
template <typename Tiles>
__device__ __forceinline__ void volume_counts(const aug_volume_desc* d, int& tiles,
                                              long long& vox) {
  constexpr bool in = tiles_over_input<Tiles>::value;
  const int onx = in ? d->in_nx : d->out_nx, ony = in ? d->in_ny : d->out_ny,
            onz = in ? d->in_nz : d->out_nz;
  const bool ok = onx >= 1 && ony >= 1 && onz >= 1 && onx <= MAX_DIM && ony <= MAX_DIM &&
                  onz <= MAX_DIM && (long long)onx * ony * onz < (1LL << 31);
  tiles = ok ? Tiles::tiles(onx, ony, onz) : 0;
  vox = ok ? (long long)onx * ony * onz : 0;
}

// Per-volume tile and voxel prefix sums of the chunk of cnt volumes starting
// at c0, into sm.tile_pre / sm.vox_pre (all threads of the CTA together; the
// leading barrier protects the previous chunk's readers).
template <int NW, typename Tiles>
__device__ __forceinline__ void chunk_scan(const aug_volume_desc* __restrict__ descs, int c0,
                                           int cnt, SchedSmem<NW * 32>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int t = 0;
  long long x = 0;
  if ((int)threadIdx.x < cnt) volume_counts<Tiles>(descs + c0 + threadIdx.x, t, x);
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
  __syncthreads();
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
}

// Calls body(v, local_tile, vox_offset) for every tile of this CTA, in
// increasing global order, with all threads of the CTA together (body may
// synchronise).  chunk_begin(c0, cnt) runs once per chunk before its tiles
// (all threads; may synchronise), e.g. to zero per-volume partial sums.
//
// The CTAs take a chunk's T tiles round-robin, CTA rank r taking tiles r,
// r + A, r + 2A, ...; the ranks rotate from chunk to chunk (rank 0 is the CTA
// after the previous chunk's last worker).  Plain order (BAL = false): A = G,
// all CTAs.  Balanced order: the chunk takes k = ceil(T / G) rounds and only
// A = ceil(T / k) CTAs work on it, each on k or k - 1 tiles; with the plain
// order T = 3.2 G leaves a fourth round of 0.2 G tiles on a fifth of the CTAs,
// a tail in which each SM holds two or three working CTAs instead of ten.
// The balanced order pays for memory-bound passes with many CTAs per SM; a
// latency-bound kernel loses more from the fewer working CTAs.  Either
// assignment depends only on T and G, so per-CTA partial sums keep a fixed
// summation order.
template <int NW, typename Tiles, bool BAL = false, typename ChunkF, typename BodyF>
__device__ __forceinline__ void for_each_tile_t(const aug_volume_desc* __restrict__ descs,
                                                int n_vols, SchedSmem<NW * 32>& sm,
                                                ChunkF&& chunk_begin, BodyF&& body) {
  constexpr int BLOCK = NW * 32;
  const long long G = gridDim.x;
  long long rot = 0;      // CTA of rank 0 in the current chunk
  long long voxbase = 0;  // output voxels before the chunk
  for (int c0 = 0; c0 < n_vols; c0 += BLOCK) {
    const int cnt = min(BLOCK, n_vols - c0);
    chunk_scan<NW, Tiles>(descs, c0, cnt, sm);
    chunk_begin(c0, cnt);
    const long long chunk_tiles = sm.tile_pre[cnt];
    if (chunk_tiles > 0) {
      const long long rounds = (chunk_tiles + G - 1) / G;
      const long long active = BAL ? (chunk_tiles + rounds - 1) / rounds : G;
      const long long r = ((long long)blockIdx.x - rot + G) % G;
      int vi = 0;
      if (r < active) {
        for (long long lt = r; lt < chunk_tiles; lt += active) {
          while (sm.tile_pre[vi + 1] <= (int)lt) ++vi;
          body(c0 + vi, (int)lt - sm.tile_pre[vi], voxbase + sm.vox_pre[vi]);
        }
      }
      rot = (rot + (BAL ? active : chunk_tiles)) % G;
    }
    voxbase += sm.vox_pre[cnt];
  }
}

template <int NW, int QZ, bool FLAT = false, bool BAL = false, typename ChunkF, typename BodyF>
__device__ __forceinline__ void for_each_tile(const aug_volume_desc* __restrict__ descs,
                                              int n_vols, SchedSmem<NW * 32>& sm,
                                              ChunkF&& chunk_begin, BodyF&& body) {
  for_each_tile_t<NW, StdTiles<NW, QZ, FLAT>, BAL>(descs, n_vols, sm, chunk_begin, body);
}

// Dynamic form of for_each_tile (same global tile order, same body
// arguments): CTA b of G starts with global tile b, and whenever it finishes
// a tile takes the next unclaimed one, (*counter)++ (*counter is G at launch),
// so CTAs that drew cheap tiles take more of them and all finish
// within about one tile of each other.  The index of the following tile is
// claimed while the current one is processed (its latency is hidden), and
// tiles are claimed in increasing order, so the tiles in flight at any time
// are neighbours, as in the static order.  A CTA without a first tile exits
// without touching the counter.  Every thread of the CTA calls body with the
// same arguments; body may synchronise the CTA, but must not use sm.
template <int NW, typename Tiles, typename BodyF>
__device__ __forceinline__ void for_each_tile_dynamic_t(const aug_volume_desc* __restrict__ descs,
                                                        int n_vols, SchedSmem<NW * 32>& sm,
                                                        unsigned long long* counter,
                                                        BodyF&& body) {
  constexpr int BLOCK = NW * 32;
  if (threadIdx.x == 0) sm.next = blockIdx.x;
  __syncthreads();
  long long g = sm.next;  // same value in every thread: the loops below are uniform
  int c0 = -BLOCK, cnt = 0, vi = 0;
  long long gbase = 0, gend = 0, voxbase = 0, chunk_vox = 0;
  while (true) {
    while (g >= gend) {
      c0 += BLOCK;
      if (c0 >= n_vols) return;
      cnt = min(BLOCK, n_vols - c0);
      gbase = gend;
      voxbase += chunk_vox;
      chunk_scan<NW, Tiles>(descs, c0, cnt, sm);
      gend = gbase + sm.tile_pre[cnt];
      chunk_vox = sm.vox_pre[cnt];
      vi = 0;
    }
    long long claimed = 0;
    if (threadIdx.x == 0) claimed = (long long)atomicAdd(counter, 1ull);
    const int lt = (int)(g - gbase);
    while (sm.tile_pre[vi + 1] <= lt) ++vi;
    body(c0 + vi, lt - sm.tile_pre[vi], voxbase + sm.vox_pre[vi]);
    __syncthreads();  // every thread is done with sm for this tile
    if (threadIdx.x == 0) sm.next = claimed;
    __syncthreads();
    g = sm.next;
  }
}

template <int NW, int QZ, bool FLAT, typename BodyF>
__device__ __forceinline__ void for_each_tile_dynamic(const aug_volume_desc* __restrict__ descs,
                                                      int n_vols, SchedSmem<NW * 32>& sm,
                                                      unsigned long long* counter,
                                                      BodyF&& body) {
  for_each_tile_dynamic_t<NW, StdTiles<NW, QZ, FLAT>>(descs, n_vols, sm, counter, body);
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
                          WsHeader* ws, unsigned long long tile_next0);

}  // namespace augk
