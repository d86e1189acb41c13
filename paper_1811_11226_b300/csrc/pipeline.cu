// Forward augmentation from host buffers, pipelined (the host <-> device FIFO
// of Sec. 4, which overlaps the transfer of the next job with the compute of
// the current one).
//
// The batch is cut into chunks of volumes.  Chunk c runs on internal stream
// c mod 3 in device slot c mod 3: its descriptors and inputs are copied to the
// device, the batched forward kernel runs, and the outputs are copied back.
// Stream order makes a slot's buffers reusable once its previous chunk's output
// copies are done; across the three streams the input copy of one chunk, the
// kernel of another and the output copy of a third run at the same time (the
// copy engines of the two directions are independent).  The caller's stream
// orders the whole call: the internal streams start after its prior work and
// it waits for them at the end.
//
// Device memory for the slots comes from the stream-ordered pool and is given
// back at the end of the call; descriptor staging uses a page-locked host
// array kept by the library per device (grown on demand).
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace augk {
namespace {

constexpr int kSlots = 3;

struct PipeState {
  std::mutex mu;
  cudaStream_t st[kSlots] = {};
  cudaEvent_t done[kSlots] = {};
  cudaEvent_t ready = nullptr;
  aug_volume_desc* h_stage = nullptr;  // page-locked descriptor staging
  size_t h_cap = 0;                    // descriptors
};

std::mutex g_pipe_mu;
std::map<int, PipeState*> g_pipe;

cudaError_t pipe_state(PipeState** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  auto it = g_pipe.find(dev);
  if (it != g_pipe.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  PipeState* P = new PipeState;
  for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&P->st[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ready, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;  // (the partial state is kept out of the map)
  g_pipe[dev] = P;
  *out = P;
  return cudaSuccess;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t in_bytes(const aug_volume_desc& d) {
  return (size_t)d.in_nx * d.in_ny * d.in_nz * (d.image_dtype == AUG_I16 ? 2 : 4);
}
size_t in_vox(const aug_volume_desc& d) { return (size_t)d.in_nx * d.in_ny * d.in_nz; }
size_t out_vox(const aug_volume_desc& d) { return (size_t)d.out_nx * d.out_ny * d.out_nz; }

// Device bytes of one chunk's slot: descriptors, forward workspace, and per
// volume its image, label, output image and output label (each 256-aligned).
size_t chunk_bytes(const aug_volume_desc* h, int n, size_t ws) {
  size_t b = up256((size_t)n * sizeof(aug_volume_desc)) + up256(ws);
  for (int v = 0; v < n; ++v) {
    if (h[v].out_image) b += up256(in_bytes(h[v])) + up256(out_vox(h[v]) * 4);
    if (h[v].out_label) b += up256(in_vox(h[v])) + up256(out_vox(h[v]));
  }
  return b;
}

}  // namespace

aug_status fwd_host_pipeline(const aug_volume_desc* h, int n, uint64_t seed, int chunk,
                             cudaStream_t stream) {
  PipeState* P = nullptr;
  if (pipe_state(&P) != cudaSuccess) return AUG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(P->mu);
  const int n_chunks = (n + chunk - 1) / chunk;
  const size_t ws = fwd_workspace_bytes(chunk);
  size_t slot = 0;
  for (int c = 0; c < n_chunks; ++c) {
    const int k = std::min(chunk, n - c * chunk);
    slot = std::max(slot, chunk_bytes(h + c * chunk, k, ws));
  }
  // A previous call's descriptor copies may still read the staging array.
  for (int s = 0; s < kSlots; ++s)
    if (cudaEventSynchronize(P->done[s]) != cudaSuccess) return AUG_ERR_CUDA;
  // Page-locked staging for every chunk's device descriptors (each copy reads
  // its own part, so no part is rewritten while a copy may still read it).
  if (P->h_cap < (size_t)n) {
    if (P->h_stage) cudaFreeHost(P->h_stage);
    P->h_stage = nullptr;
    P->h_cap = 0;
    if (cudaMallocHost((void**)&P->h_stage, (size_t)n * sizeof(aug_volume_desc)) != cudaSuccess)
      return AUG_ERR_CUDA;
    P->h_cap = (size_t)n;
  }

  const int n_slots = std::min(kSlots, n_chunks);
  char* buf[kSlots] = {};
  for (int s = 0; s < n_slots; ++s) {
    if (cudaMallocAsync((void**)&buf[s], slot, stream) != cudaSuccess) {
      for (int t = 0; t < s; ++t) cudaFreeAsync(buf[t], stream);
      return AUG_ERR_CUDA;
    }
  }
  cudaError_t e = cudaEventRecord(P->ready, stream);
  for (int s = 0; s < n_slots && e == cudaSuccess; ++s) {
    e = cudaStreamWaitEvent(P->st[s], P->ready, 0);
    // The workspace's status header starts cleared.
    char* wsp = buf[s] + up256((size_t)chunk * sizeof(aug_volume_desc));
    if (e == cudaSuccess) e = cudaMemsetAsync(wsp, 0, 256, P->st[s]);
  }

  for (int c = 0; c < n_chunks && e == cudaSuccess; ++c) {
    const int s = c % kSlots, v0 = c * chunk, k = std::min(chunk, n - v0);
    cudaStream_t st = P->st[s];
    char* base = buf[s];
    aug_volume_desc* d_desc = (aug_volume_desc*)base;
    void* d_ws = base + up256((size_t)chunk * sizeof(aug_volume_desc));
    char* p = (char*)d_ws + up256(ws);
    aug_volume_desc* hd = P->h_stage + v0;
    // Device layout of the chunk; inputs go up while the descriptors are built.
    for (int v = 0; v < k && e == cudaSuccess; ++v) {
      const aug_volume_desc& src = h[v0 + v];
      aug_volume_desc d = src;
      if (src.out_image) {
        d.image = p;
        e = cudaMemcpyAsync(p, src.image, in_bytes(src), cudaMemcpyHostToDevice, st);
        p += up256(in_bytes(src));
        d.out_image = (float*)p;
        p += up256(out_vox(src) * 4);
      } else {
        d.image = nullptr;
      }
      if (src.out_label && e == cudaSuccess) {
        d.label = (const uint8_t*)p;
        e = cudaMemcpyAsync(p, src.label, in_vox(src), cudaMemcpyHostToDevice, st);
        p += up256(in_vox(src));
        d.out_label = (uint8_t*)p;
        p += up256(out_vox(src));
      } else if (!src.out_label) {
        d.label = nullptr;
      }
      hd[v] = d;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_desc, hd, (size_t)k * sizeof(aug_volume_desc),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = fwd_on_device(d_desc, k, seed, d_ws, st);
    for (int v = 0; v < k && e == cudaSuccess; ++v) {
      const aug_volume_desc& src = h[v0 + v];
      if (src.out_image)
        e = cudaMemcpyAsync(src.out_image, hd[v].out_image, out_vox(src) * 4,
                            cudaMemcpyDeviceToHost, st);
      if (src.out_label && e == cudaSuccess)
        e = cudaMemcpyAsync(src.out_label, hd[v].out_label, out_vox(src),
                            cudaMemcpyDeviceToHost, st);
    }
  }
  // Join: the caller's stream waits for every slot, then the slots go back to
  // the pool in its order.
  for (int s = 0; s < kSlots; ++s) {
    if (cudaEventRecord(P->done[s], P->st[s]) != cudaSuccess) e = cudaErrorUnknown;
    if (cudaStreamWaitEvent(stream, P->done[s], 0) != cudaSuccess) e = cudaErrorUnknown;
  }
  for (int s = 0; s < n_slots; ++s)
    if (cudaFreeAsync(buf[s], stream) != cudaSuccess) e = cudaErrorUnknown;
  return e == cudaSuccess ? AUG_OK : AUG_ERR_CUDA;
}

}  // namespace augk
