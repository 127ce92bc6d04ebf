// Batched fused forward for callers that cannot allocate device memory.
//
// Same persistent kernel as dwtfuse_fuse_batched, but the work-queue counter
// and the device status word live in a file-scope device array that the
// library owns, instead of in a caller workspace.  The array is created when
// the library's device code is loaded on a GPU and lives until the process
// exits; nothing here calls cudaMalloc, cudaFree or an allocating library
// routine.
#include <cstring>
#include <mutex>

#include "dwtfuse.h"
#include "launch.h"

namespace dwtfuse {

// Defined in api.cu.
int build_batch_table(const dwtfuse_scene *scenes, int n, int rows_per_item, BatchTable *t);
int cuda_status(cudaError_t e);

namespace {

// Queue counter (bytes 0-7) and status word (bytes 8-11) of one batched launch.
static __device__ __align__(256) unsigned char g_batched_scratch[DWTFUSE_STATIC_SCRATCH_BYTES];
static_assert(kQueueBytes <= DWTFUSE_STATIC_SCRATCH_BYTES, "static scratch too small for the queue");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_batched_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device with that device current, and cached.
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return DWTFUSE_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_batched_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return DWTFUSE_OK;
}

}  // namespace

// Status word of the last dwtfuse_fuse_batched_noalloc call on the current
// device, read synchronously on `stream` (a copy from the static array;
// nothing is allocated).
int noalloc_device_status(cudaStream_t stream) {
    void *scratch = nullptr;
    const int st = scratch_address(&scratch);
    if (st != DWTFUSE_OK) return st;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, static_cast<const char *>(scratch) + 8, sizeof v, cudaMemcpyDeviceToHost,
                                    stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    return v;
}

}  // namespace dwtfuse

using namespace dwtfuse;

extern "C" int dwtfuse_fuse_batched_noalloc(const dwtfuse_scene *scenes, int n, int rows_per_item,
                                            int blocks_per_sm, void *stream) {
    if (!scenes || n < 1 || rows_per_item < 0 || blocks_per_sm < 0) return DWTFUSE_EINVAL;
    if (n > kMaxScenes) return DWTFUSE_ESHAPE;
    static thread_local BatchTable t;
    int st = build_batch_table(scenes, n, rows_per_item, &t);
    if (st != DWTFUSE_OK) return st;
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != DWTFUSE_OK) return st;
    // launch_fuse_batched clears the counter and status word before the kernel.
    auto *queue = static_cast<unsigned long long *>(scratch);
    int *status = reinterpret_cast<int *>(static_cast<char *>(scratch) + 8);
    return cuda_status(launch_fuse_batched(t, queue, status, blocks_per_sm, static_cast<cudaStream_t>(stream)));
}
