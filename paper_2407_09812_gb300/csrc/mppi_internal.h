// Internal declarations shared by the CUDA kernels, the C ABI and the
// serving runtime.  Nothing here is part of the public ABI (include/mppi.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mppi.h"

#ifdef __CUDACC__
#define MPPI_HD __host__ __device__
#else
#define MPPI_HD
#endif

namespace mppi {

// Vehicle model in the form the kernels use (derived on the host, FP64,
// then rounded once to FP32).
struct DevModel {
    float inv_mass, g;
    float Jx, Jy, Jz;
    float inv_Jx, inv_Jy, inv_Jz;
    float dJx, dJy, dJz;    // (Jz-Jy), (Jx-Jz), (Jy-Jx): omega x J omega terms
    float kx, ky, kz;       // dJ / J: gyroscopic angular-acceleration factors
    float a, c_tf;          // a = l / sqrt(2): entries of the allocation matrix
    float T_min, T_max;
    int motor_clip;
    float F_min, F_max;
    float w_max[3];
    float u_init[4];        // hover: m g, 0, 0, 0
    // Motor allocation in factored form (Gamma's rows are (1,1,1,1),
    // a(-1,1,1,-1), a(-1,1,-1,1), c(-1,-1,1,1)): rotor thrusts from
    // F/4 and the torques times q_a = 1/(4a), q_c = 1/(4c); torque over
    // inertia from the clipped thrusts' differences times a/J_x, a/J_y, c/J_z.
    float q_a, q_c;
    float a_Jx, a_Jy, c_Jz;
};

// Cost weights and step options shared by every instance of a launch.
// A warp's kept-obstacle list is built for the warp's position box grown by
// this margin on every side and reused while all of the warp's positions stay
// inside; a larger margin means fewer rebuilds but more (exactly zero) terms.
// The pipelined form, whose cost lanes wait on the list, is faster with the
// smaller margin (closed-loop step, 64 spheres: 91 against 93 us).
constexpr float kCullMargin = 1.0f;           // [m]
constexpr float kCullMarginPipelined = 0.5f;  // [m]

// Floor of the obstacle barrier: a term exp(-beta max(s, 0)) below
// 2^-kBarrierFloorLog2 counts as exactly zero.  Per obstacle and state that
// drops at most 2^-48 c_bar (3.6e-13 at c_bar = 100), far below the FP32
// resolution of any rollout cost; in exchange an obstacle whose squared gap
// exceeds kBarrierFloorLog2 / (beta log2 e) (5.9 m + r at beta = 1) is
// skipped, against 9.4 m + r where the FP32 exponential itself reaches 0.
constexpr float kBarrierFloorLog2 = 48.0f;

struct DevCost {
    float c_p, c_q, c_v, c_w;
    float R[4], Rd[4];
    float c_obs, c_bar, beta_log2e, r_uav;
    float cull;             // squared gap beyond which the barrier term is below its floor (counts as 0)
    float cull_margin;      // enlargement of a warp's box when its kept-obstacle list is built [m]
    int quat_metric, tail_mode;
    float shift_alpha, delay;
    // Occupancy voxel grid (NULL: none): grid[(iz*gy + iy)*gx + ix] != 0 is
    // occupied; voxel (ix, iy, iz) spans origin + voxel * [i, i+1).
    const unsigned char* grid;
    int gx, gy, gz;
    float g_origin[3];
    float g_inv_voxel;
};

// One instance (vehicle problem) of a launch.
struct DevInstance {
    const float* x_hat;
    const float* ref;
    const float4* obs;
    const float* u_nom;
    float* u_out;
    float* u_cmd;
    float* u_next;
    float* x_next;
    float* costs;
    int* status;
    unsigned long long* iter_dev;
    unsigned long long iter;
    long long part_off;     // float offset of this instance's first tile partial
    int K, N, M, n_tiles;
    float dt, lambda;
    float sigma[4];
    unsigned key0, key1;
};

struct Shape {
    int block;     // threads per block
    int lanes;     // lanes per sample
    int pipe;      // 1: pipelined (a dynamics thread and cost lanes per sample); 2: also a noise thread;
                   // 3: also the dynamics split into attitude and translation threads
    float margin;  // kept-obstacle list margin [m]; 0: the default of the form
    int spt = 1;   // samples per thread (2: pipe 0, lanes 1, blocks of 64 or 128 threads)
};

// Samples a block of this shape rolls out (the tile size).
inline int samples_per_block(const Shape& s) {
    return s.pipe ? s.block / (s.pipe + s.lanes) : s.spt * s.block / s.lanes;
}

inline float list_margin(const Shape& s) {
    return s.margin > 0.0f ? s.margin : s.pipe ? kCullMarginPipelined : kCullMargin;
}

// Everything one launch of the fused kernel needs.
struct LaunchArgs {
    const DevInstance* insts;   // device array; NULL: the single instance below
    const int2* tile_map;       // (instance, tile) per global tile; NULL: (0, t)
    unsigned* tile_counter;     // dynamic tile scheduler; NULL: one tile per block
    float* partials;            // per-tile (rho_t, eta_t, s_t, Sigma_t)
    unsigned* done;             // per-instance count of finished tiles
    unsigned* errflags;         // per-instance error bits
    const int* n_tiles_dev;     // device tile count (graph replay); NULL: n_tiles
    unsigned long long* stats;  // optional: [0] += evaluated (state, obstacle) pairs
    long long wait_polls;       // bound of every device-side wait (polls); 0: default
    int stall_obstacle_copy;    // test hook: skip the obstacle copy so its wait runs out
    int n_tiles;
    int n_inst;
    int N_max, M_max;           // sizes the dynamic shared memory was laid out for
    DevModel M;
    DevCost C;
    DevInstance single;
};

constexpr unsigned ERR_TIMEOUT = 1u;

// Floats of one tile partial: rho_t (a cost pair hi, lo), eta_t, the merge
// scale s_t, then Sigma_t[N][4].
MPPI_HD inline int partial_stride(int N) { return 4 + 4 * N; }

// Host-side validation and conversion of the public parameter structs.
int check_model(const mppi_model* m);
int check_params(const mppi_params* p);
int check_step(int K, int N, float dt, float lambda, const float* sigma);
DevModel make_dev_model(const mppi_model& m);
DevCost make_dev_cost(const mppi_params& p);
bool aligned16(const void* p);
bool aligned4(const void* p);

size_t smem_bytes(int N_max, int M_max, Shape s);
// Largest dynamic shared memory a launch may request: the 227 KB a block can
// address less room for the kernel's static shared memory (under 8 KB in
// every instantiation).
constexpr size_t kMaxDynamicSmem = 227 * 1024 - 8 * 1024;
bool shape_supported(Shape s);
cudaError_t launch_tiles(const LaunchArgs& a, Shape s, int grid, size_t smem, cudaStream_t st);
int max_active_blocks(Shape s, size_t smem);
int sm_count();
// delta of samples k0 .. k0 + K - 1, steps 0 .. N - 1 into out (16-byte aligned, K N float4).
cudaError_t launch_noise(float* out, unsigned k0, int K, int N, unsigned long long iter, unsigned key0,
                         unsigned key1, const float* sigma, cudaStream_t st);

}  // namespace mppi
