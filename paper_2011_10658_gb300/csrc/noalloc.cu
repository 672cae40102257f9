// y = H_eff x at a bottom-node centre without any memory allocation.
//
// Who needs this: a caller whose device memory belongs to someone else --
// a serving runtime or framework that hands every buffer out of its own
// pool or of an arena fixed at start-up -- and that therefore cannot let a
// library call cudaMalloc or cudaFree (which also synchronise the whole
// device).  The caller passes x and y; everything else this product needs
// beyond them lives in one file-scope device array of fixed size.
//
// It is a variant of the product ttn_apply_heff_device computes with the
// FP64 grouped-GEMM kernel: the work list of that kernel (tiles, outputs,
// term chunks) and any split-K partial sums are the scratch, and here they
// are placed in g_heff_scratch instead of buffers the state allocates.  The
// work list is written on the host into a fixed static buffer first, so no
// host allocation happens either.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/qedttn.h"
#include "engine.h"
#include "kernels.cuh"
#include "state.h"

namespace {

// 4 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = size_t(4) << 20;
// regions of the array: tiles, outputs, chunks
constexpr size_t kTileBytes = size_t(5) << 19;     // 2.5 MiB
constexpr size_t kOutBytes = size_t(1) << 18;      // 0.25 MiB
constexpr size_t kChunkBytes = kScratchBytes - kTileBytes - kOutBytes;

static __device__ __align__(256) unsigned char g_heff_scratch[kScratchBytes];

// Device address of g_heff_scratch per device (the host-side name is only a
// stand-in and must never be passed to a kernel).
constexpr int kMaxDevices = 64;
void* g_dev_addr[kMaxDevices] = {};
std::mutex g_mu;
alignas(256) unsigned char g_host[kScratchBytes];

int fail(int code, const char* msg) {
  qed_set_last_error(msg);
  return code;
}

}  // namespace

#define QED_API __attribute__((visibility("default")))

extern "C" {

QED_API int ttn_apply_heff_device_noalloc(ttn_state* s, const double* x_device, double* y_device, int64_t n) {
  if (!s || !x_device || !y_device) return fail(QED_EINVAL, "null argument");
  qed::Engine* e = s->engine;
  if (n != e->node_size(e->center())) return fail(QED_EINVAL, "size must equal the centre tensor size");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(QED_ECUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_addr[dev]) {
    // once per device, with that device current
    void* ptr = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&ptr, g_heff_scratch);
    if (err != cudaSuccess || !ptr) return fail(QED_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    g_dev_addr[dev] = ptr;
  }
  unsigned char* dbase = (unsigned char*)g_dev_addr[dev];
  qed::KTile* tiles = (qed::KTile*)g_host;
  qed::KOutput* outs = (qed::KOutput*)(g_host + kTileBytes);
  qed::KChunk* chunks = (qed::KChunk*)(g_host + kTileBytes + kOutBytes);
  int nt = 0, no = 0, nc = 0;
  int rc = e->noalloc_worklist(x_device, y_device, tiles, (int)(kTileBytes / sizeof(qed::KTile)), outs,
                               (int)(kOutBytes / sizeof(qed::KOutput)), chunks,
                               (int)(kChunkBytes / sizeof(qed::KChunk)), &nt, &no, &nc);
  if (rc == -2) return fail(QED_EUNSUPPORTED, "work list exceeds the 4 MiB scratch array");
  // the engine names what is missing: a centre that is not a bottom node, or
  // a row map / environment operator not built yet at this centre
  if (rc) return fail(QED_EUNSUPPORTED, e->error().c_str());
  cudaStream_t st = e->stream();
  // the whole work list is rewritten every call; nothing must start at zero
  // (every output tile is stored, not accumulated, and no partial sums are used).
  // g_host is pageable: a host-to-device cudaMemcpyAsync from pageable memory
  // first waits for the work already queued on the stream and returns once
  // the host buffer has been read, so the next call may rewrite g_host.
  if (cudaMemcpyAsync(dbase, tiles, nt * sizeof(qed::KTile), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dbase + kTileBytes, outs, no * sizeof(qed::KOutput), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(dbase + kTileBytes + kOutBytes, chunks, nc * sizeof(qed::KChunk), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return fail(QED_ECUDA, "copy of the work list failed");
  qed::launch_kc_gemm((const qed::KTile*)dbase, nt, (const qed::KOutput*)(dbase + kTileBytes),
                      (const qed::KChunk*)(dbase + kTileBytes + kOutBytes), nullptr, st, 0);
  if (cudaGetLastError() != cudaSuccess) return fail(QED_ECUDA, "kernel launch failed");
  return QED_OK;
}

}  // extern "C"
