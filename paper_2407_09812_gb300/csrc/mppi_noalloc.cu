// mppi_solve_noalloc: one MPPI step that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code running under a real-time
// control loop that forbids allocation after start-up (allocation can
// block for an unbounded time and fragment device memory), plug-ins that
// live inside a host framework which owns all device memory, and callers
// whose device memory is fully reserved by another allocator.  A handle
// (mppi_create) allocates its workspace, so those callers cannot use it.
// This entry point runs the same fused kernel with its scratch (the tile
// partials and the per-instance completion counters) in a fixed array
// compiled into this file instead.  The caller still passes every input
// and output buffer.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it (about 1 MiB) until the process exits.  In host code its
// name is only a host-side stand-in, so its device address is looked up
// with cudaGetSymbolAddress, once per device, on the first call made with
// that device current; that first call should therefore come before any
// stream capture.  The looked-up address is kept for the life of the
// process and is not valid after the device's primary context is torn
// down (cudaDeviceReset).  All calls share the array and it keeps the last call's
// contents: each call clears the counters that must start at zero, and
// calls whose work overlaps on the GPU (different streams, no ordering)
// race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "mppi_internal.h"

using namespace mppi;

namespace {

// Largest problem the fixed scratch serves: K <= 32768 samples and
// N <= 256 steps (256 tiles of 128 samples, 4 + 4N floats each), plus a
// 256-byte header for the completion counter and the error flag.
constexpr int kNoAllocBlock = 128;
constexpr int kNoAllocMaxK = 32768;
constexpr int kNoAllocMaxN = 256;
constexpr int kNoAllocMaxTiles = kNoAllocMaxK / kNoAllocBlock;
constexpr int kHeaderFloats = 64;
constexpr size_t kScratchFloats = kHeaderFloats + (size_t)kNoAllocMaxTiles * (4 + 4 * kNoAllocMaxN);

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up
// once per device).
int scratch_for_current_device(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MPPI_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MPPI_ECUDA;
        }
        g_scratch_dev[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_dev[dev];
    return MPPI_OK;
}

}  // namespace

extern "C" int mppi_solve_noalloc(const mppi_model* model, const mppi_params* params, const float* x_hat,
                                  const float* ref, const float* obstacles, int32_t M, const float* u_nom,
                                  uint64_t iter, float* u_out, float* u_cmd, float* u_next, float* x_next,
                                  float* costs, int32_t* status, void* stream) {
    int rc = check_model(model);
    if (rc) return rc;
    if ((rc = check_params(params))) return rc;
    if (params->K > kNoAllocMaxK || params->N > kNoAllocMaxN) return MPPI_EINVAL;
    if (!x_hat || !ref || !u_nom || M < 0 || M > MPPI_M_MAX) return MPPI_EINVAL;
    if (M > 0 && (!obstacles || !aligned16(obstacles))) return MPPI_EINVAL;
    // The kernel reads and writes these with 4-byte accesses: a misaligned
    // pointer would fault on the device, so it is refused here.
    const void* ptrs[] = {x_hat, ref, u_nom, u_out, u_cmd, u_next, x_next, costs, status};
    for (const void* p : ptrs)
        if (p && !aligned4(p)) return MPPI_EINVAL;

    const Shape shape{kNoAllocBlock, 1};
    const size_t smem = smem_bytes(params->N, M, shape);
    if (smem > kMaxDynamicSmem) return MPPI_EINVAL;

    float* scratch = nullptr;
    if ((rc = scratch_for_current_device(&scratch))) return rc;
    unsigned* counters = reinterpret_cast<unsigned*>(scratch);  // [0] done, [1] error flags
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned), st) != cudaSuccess) {
        cudaGetLastError();
        return MPPI_ECUDA;
    }

    DevInstance d = {};
    d.x_hat = x_hat;
    d.ref = ref;
    d.obs = reinterpret_cast<const float4*>(obstacles);
    d.u_nom = u_nom;
    d.u_out = u_out;
    d.u_cmd = u_cmd;
    d.u_next = u_next;
    d.x_next = x_next;
    d.costs = costs;
    d.status = status;
    d.iter = iter;
    d.part_off = 0;
    d.K = params->K;
    d.N = params->N;
    d.M = M;
    d.n_tiles = (params->K + kNoAllocBlock - 1) / kNoAllocBlock;
    d.dt = params->dt;
    d.lambda = params->lambda;
    for (int c = 0; c < 4; ++c) d.sigma[c] = params->sigma[c];
    d.key0 = (unsigned)(params->seed & 0xffffffffu);
    d.key1 = (unsigned)(params->seed >> 32) ^ params->stream_id;

    LaunchArgs a = {};
    a.partials = scratch + kHeaderFloats;
    a.done = counters;
    a.errflags = counters + 1;
    a.n_tiles = d.n_tiles;
    a.n_inst = 1;
    a.N_max = params->N;
    a.M_max = M;
    a.M = make_dev_model(*model);
    a.C = make_dev_cost(*params);
    a.single = d;
    return launch_tiles(a, shape, d.n_tiles, smem, st) == cudaSuccess ? MPPI_OK : MPPI_ECUDA;
}
