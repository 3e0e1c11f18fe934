// Fused MPPI step kernel for sm_103a.
//
// One launch computes, for one or many independent instances (vehicles),
// the whole MPPI iteration of Alg. 1:
//   * noise delta u_j^k ~ N(0, Sigma) from a counter-based Philox4x32-10
//     generator inside the kernel (Sec. III-A, Eq. rollout_computation),
//     regenerated rather than stored;
//   * the rollout x_{j+1} = x_j + f_RK4(x_j, u_j, dt) of Eq. drone_dynamics
//     with the motor-constraint pipeline of Sec. III-B, state in registers;
//   * the tracking / input / input-change cost of Sec. IV-C and the
//     obstacle cost of Sec. IV-D fused into the rollout, obstacles staged
//     in shared memory by a bulk TMA copy;
//   * per tile of samples: warp-shuffle min, min-shifted exponential
//     weights (Eq. cost_2) and the weighted sum of the regenerated noise;
//   * the last block of an instance merges the tile partials in a fixed
//     order (log-sum-exp rescaling), applies Eq. u_update, computes the
//     command sent to the low-level controller and the warm-start shift.
//
// Tiles are (instance, block of samples).  A persistent grid pulls tiles
// from an atomic counter (batched launches) or each block takes one tile
// (single instance).  The per-instance result depends only on the
// instance and the launch shape, never on what else is in the launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "mppi_internal.h"

namespace mppi {

// ------------------------------------------------------------------ noise

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the multiply/xor
// network; round r uses the key (k0 + r W0, k1 + r W1), W the Weyl
// constants.  The round keys are the same for every sample of an instance,
// so they are formed once per tile (philox_round_keys) and read from shared
// memory as five (round 2i, round 2i + 1) pairs.
constexpr unsigned kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Packed FP32x2 arithmetic (two lanes' worth of work per instruction, each
// element rounded as the scalar operation; the assembler may still fuse a
// packed multiply into a following packed add, explicit rounding mode or
// not, so a sequence of packed operations is exact to FP32 rounding, not
// necessarily bitwise equal to the same sequence written with scalar
// intrinsics).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}


__device__ __forceinline__ uint4 philox_round(uint4 c, unsigned k0, unsigned k1) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z);
    const unsigned lo1 = 0xCD9E8D57u * c.z;
    return make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
}

__device__ __forceinline__ uint4 philox_round_keys(unsigned key0, unsigned key1, unsigned i) {
    return make_uint4(key0 + 2u * i * kPhiloxW0, key1 + 2u * i * kPhiloxW1, key0 + (2u * i + 1u) * kPhiloxW0,
                      key1 + (2u * i + 1u) * kPhiloxW1);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint4* rk) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint4 k = rk[i];
        c = philox_round(c, k.x, k.y);
        c = philox_round(c, k.z, k.w);
    }
    return c;
}

// Uniform in (0, 1) from the top 23 bits m: (2m + 1) 2^-24, exact in FP32.
// Formed as (1 + m 2^-23) - (1 - 2^-24): the first operand is m placed in
// the mantissa of 1.0, both operands and the difference are FP32 numbers,
// so the subtraction is exact (no integer-to-float conversion).
__device__ __forceinline__ float uniform01(unsigned r) {
    return __uint_as_float(0x3f800000u | (r >> 9)) - 0.99999994039535522f;
}

// -2 ln u for u of the map above, u in [2^-24, 1 - 2^-24].  Away from 1 it
// is -2 ln 2 log2(u) with the hardware log2 (lg2.approx: absolute error
// about 2^-22 for u in [0.5, 1), a few ulp below); for d = 1 - u <= 2^-6
// (d exact there), where an absolute error in log2 would dominate the small
// result, it is the Mercator series -2 ln(1 - d) = 2 (d + d^2/2 + d^3/3 +
// d^4/4 + ...) to the fourth term, whose truncation is below d^4/5 <= 2^-24
// relative.  Measured over all 2^23 values of the map: relative error of
// -2 ln u at most 2.4e-6 and of its square root (the Box-Muller radius) at
// most 1.3e-6, absolute 7.2e-7 (the square root by x rsqrt(x)).
__device__ __forceinline__ float neg2log(float u) {
    float l;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(u));
    const float far = -1.3862943611198906f * l;
    const float d = 1.0f - u;
    const float near = d * fmaf(d, fmaf(d, fmaf(d, 0.5f, 0.66666669f), 1.0f), 2.0f);
    return d <= 0.015625f ? near : far;
}

// Box-Muller on the two uniform pairs of one Philox output.
__device__ __forceinline__ float4 box_muller4(const uint4 r) {
    const float u0 = uniform01(r.x), u1 = uniform01(r.y), u2 = uniform01(r.z), u3 = uniform01(r.w);
    // neg2log > 0 over the whole map (u < 1), so sqrt(x) = x rsqrt(x).
    const float a01 = neg2log(u0), a23 = neg2log(u2);
    const float rad01 = a01 * rsqrtf(a01);
    const float rad23 = a23 * rsqrtf(a23);
    // Angle 2 pi u taken as 2 pi u - pi in (-pi, pi), where the hardware
    // sine/cosine are accurate to ~5e-7 absolute; cos and sin change sign.
    const float t1 = fmaf(6.2831853071795865f, u1, -3.1415926535897932f);
    const float t3 = fmaf(6.2831853071795865f, u3, -3.1415926535897932f);
    float s1, c1, s3, c3;
    __sincosf(t1, &s1, &c1);
    __sincosf(t3, &s3, &c3);
    return make_float4(-rad01 * c1, -rad01 * s1, -rad23 * c3, -rad23 * s3);
}

// Four standard normals for sample k, step j: Box-Muller on the two
// uniform pairs of one Philox call.  Counter (k, j, iter), round keys rk.
__device__ __forceinline__ float4 normals4(unsigned k, unsigned j, unsigned long long iter, const uint4* rk) {
    return box_muller4(philox4x32_10(make_uint4(k, j, (unsigned)iter, (unsigned)(iter >> 32)), rk));
}

// The first round's output words that do not depend on the step j: two
// that depend on the sample k only (and the counter's high word), two on
// the tile's counter word only.  normals4_pre gives bitwise normals4.
struct PhiloxPre {
    unsigned z, w;  // per sample: mulhi(M0, k) ^ iter_hi ^ key1, M0 k
};

__device__ __forceinline__ PhiloxPre philox_pre_sample(unsigned k, unsigned long long iter, const uint4* rk) {
    PhiloxPre p;
    p.z = __umulhi(0xD2511F53u, k) ^ (unsigned)(iter >> 32) ^ rk[0].y;
    p.w = 0xD2511F53u * k;
    return p;
}

// Per tile: (mulhi(M1, iter_lo) ^ key0, M1 iter_lo).
__device__ __forceinline__ uint2 philox_pre_tile(unsigned long long iter, const uint4* rk) {
    const unsigned lo = (unsigned)iter;
    return make_uint2(__umulhi(0xCD9E8D57u, lo) ^ rk[0].x, 0xCD9E8D57u * lo);
}

// The Philox output for step j from the precomputed first-round words.
__device__ __forceinline__ uint4 philox_pre(unsigned j, const PhiloxPre p, const uint2* pt, const uint4* rk) {
    const uint2 t = *pt;
    uint4 c = make_uint4(t.x ^ j, t.y, p.z, p.w);
    c = philox_round(c, rk[0].z, rk[0].w);
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        const uint4 k = rk[i];
        c = philox_round(c, k.x, k.y);
        c = philox_round(c, k.z, k.w);
    }
    return c;
}

__device__ __forceinline__ float4 normals4_pre(unsigned j, const PhiloxPre p, const uint2* pt, const uint4* rk) {
    return box_muller4(philox_pre(j, p, pt, rk));
}

// delta = sigma o z, rounded once (no contraction) so that the rollout and
// the regeneration in the weighted sum see the same value.
__device__ __forceinline__ float4 noise_delta(const float4 z, const float* sigma) {
    const float2 a = __fmul2_rn(f2(sigma[0], sigma[1]), f2(z.x, z.y));
    const float2 b = __fmul2_rn(f2(sigma[2], sigma[3]), f2(z.z, z.w));
    return make_float4(a.x, a.y, b.x, b.y);
}

// u_nom_j + delta, rounded once per component (no contraction).
__device__ __forceinline__ float4 perturb(const float4 un, const float4 d) {
    const float2 a = __fadd2_rn(f2(un.x, un.y), f2(d.x, d.y));
    const float2 b = __fadd2_rn(f2(un.z, un.w), f2(d.z, d.w));
    return make_float4(a.x, a.y, b.x, b.y);
}

// ------------------------------------------------------------------ model

struct State {
    float px, py, pz, qw, qx, qy, qz, vx, vy, vz, wx, wy, wz;
};

// Compensated addition of inc to (x0, x1) with compensation terms (c0, c1).
__device__ __forceinline__ void comp_add2(float& x0, float& x1, float& c0, float& c1, float i0, float i1) {
    const float2 y = sub2(f2(i0, i1), f2(c0, c1));
    const float2 x = f2(x0, x1);
    const float2 t = __fadd2_rn(x, y);
    const float2 c = sub2(sub2(t, x), y);
    x0 = t.x; x1 = t.y;
    c0 = c.x; c1 = c.y;
}

// Eq. drone_dynamics split by what each part depends on: the attitude
// and body rates (q, omega) evolve on their own, given the torque over inertia
// (tJx, tJy, tJz); the acceleration depends on the attitude alone, given the
// collective thrust over mass Fm; p_dot = v.  Every operation is written out
// (fmaf, __fmul_rn), so the compiler contracts nothing and each part rounds
// identically wherever it is inlined (one thread, or the two warps of the
// split pipelined form).
struct Att {
    float qw, qx, qy, qz, wx, wy, wz;
};

__device__ __forceinline__ Att att_deriv(const DevModel& M, const Att& s, float tJx, float tJy, float tJz) {
    Att d;
    const float hx = 0.5f * s.wx, hy = 0.5f * s.wy, hz = 0.5f * s.wz;
    d.qw = fmaf(-s.qz, hz, fmaf(-s.qy, hy, __fmul_rn(-s.qx, hx)));
    d.qx = fmaf(-s.qz, hy, fmaf(s.qy, hz, __fmul_rn(s.qw, hx)));
    d.qy = fmaf(s.qz, hx, fmaf(-s.qx, hz, __fmul_rn(s.qw, hy)));
    d.qz = fmaf(-s.qy, hx, fmaf(s.qx, hy, __fmul_rn(s.qw, hz)));
    d.wx = fmaf(-__fmul_rn(M.kx, s.wy), s.wz, tJx);
    d.wy = fmaf(-__fmul_rn(M.ky, s.wz), s.wx, tJy);
    d.wz = fmaf(-__fmul_rn(M.kz, s.wx), s.wy, tJz);
    return d;
}

// Thrust along the body z axis, R(q) e_z (F/m), then gravity.
__device__ __forceinline__ float3 accel(const DevModel& M, float4 q, float Fm) {
    const float F2 = 2.0f * Fm;
    return make_float3(__fmul_rn(fmaf(q.y, q.w, __fmul_rn(q.x, q.z)), F2),
                       __fmul_rn(fmaf(q.z, q.w, -__fmul_rn(q.x, q.y)), F2),
                       fmaf(-F2, fmaf(q.y, q.y, __fmul_rn(q.z, q.z)), Fm - M.g));
}

// Low-order parts of position and velocity (compensated summation).
struct Comp {
    float px, py, pz, vx, vy, vz;
};

// Attitudes (w, x, y, z) at which RK4's second, third and fourth stages are
// evaluated.
struct Stages {
    float4 q1, q2, q3;
};

// Classical RK4 step of length h, inputs held, for the attitude and rates:
// the four stage increments are summed first and added once, then q is
// renormalised.  Returns the stage attitudes the translation part needs.
__device__ __forceinline__ Stages rk4_att(const DevModel& M, State& x, float tJx, float tJy, float tJz, float h) {
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
    const Att x0 = {x.qw, x.qx, x.qy, x.qz, x.wx, x.wy, x.wz};
    Att k = att_deriv(M, x0, tJx, tJy, tJz);
    float2 i_q0 = __fmul2_rn(f2(h6, h6), f2(k.qw, k.qx)), i_q1 = __fmul2_rn(f2(h6, h6), f2(k.qy, k.qz));
    float2 i_w = __fmul2_rn(f2(h6, h6), f2(k.wx, k.wy));
    float i_wz = h6 * k.wz;
    const float2 x_q0 = f2(x0.qw, x0.qx), x_q1 = f2(x0.qy, x0.qz), x_w = f2(x0.wx, x0.wy);
    Att xs;
    auto stage = [&](float hs) {  // xs = x + hs k
        const float2 H = f2(hs, hs);
        const float2 q0 = __ffma2_rn(H, f2(k.qw, k.qx), x_q0), q1 = __ffma2_rn(H, f2(k.qy, k.qz), x_q1);
        const float2 w = __ffma2_rn(H, f2(k.wx, k.wy), x_w);
        xs.qw = q0.x; xs.qx = q0.y; xs.qy = q1.x; xs.qz = q1.y;
        xs.wx = w.x; xs.wy = w.y; xs.wz = fmaf(hs, k.wz, x0.wz);
        return make_float4(xs.qw, xs.qx, xs.qy, xs.qz);
    };
    auto add = [&](float hc) {
        const float2 H = f2(hc, hc);
        i_q0 = __ffma2_rn(H, f2(k.qw, k.qx), i_q0);
        i_q1 = __ffma2_rn(H, f2(k.qy, k.qz), i_q1);
        i_w = __ffma2_rn(H, f2(k.wx, k.wy), i_w);
        i_wz = fmaf(hc, k.wz, i_wz);
    };
    Stages st;
    st.q1 = stage(h2);
    k = att_deriv(M, xs, tJx, tJy, tJz);
    add(h3);
    st.q2 = stage(h2);
    k = att_deriv(M, xs, tJx, tJy, tJz);
    add(h3);
    st.q3 = stage(h);
    k = att_deriv(M, xs, tJx, tJy, tJz);
    add(h6);
    float2 q0 = __fadd2_rn(x_q0, i_q0);
    float2 q1 = __fadd2_rn(x_q1, i_q1);
    const float2 w = __fadd2_rn(x_w, i_w);
    x.wx = w.x; x.wy = w.y; x.wz += i_wz;
    const float2 n2 = __ffma2_rn(q1, q1, __fmul2_rn(q0, q0));
    const float n = rsqrtf(n2.x + n2.y);
    q0 = __fmul2_rn(q0, f2(n, n));
    q1 = __fmul2_rn(q1, f2(n, n));
    x.qw = q0.x; x.qx = q0.y; x.qy = q1.x; x.qz = q1.y;
    return st;
}

// Translation part of the same RK4 step: v_dot depends on the attitude only
// and p_dot = v, so the position increment of the four stages is
// h v_0 + h^2/6 (a_1 + a_2 + a_3), a_i the stages' accelerations (the
// classical combination written out), and the velocity increment the
// classical weighted sum of a_1..a_4.  q0 is the attitude at the step's start.
// Position and velocity carry a compensation term across steps so that
// their FP32 rounding does not accumulate over the horizon.
__device__ __forceinline__ void rk4_trans(const DevModel& M, State& x, Comp& c, float4 q0, const Stages& st, float Fm,
                                          float h) {
    const float h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f), hh6 = h * h6;
    float3 a = accel(M, q0, Fm);
    float ax = a.x, ay = a.y, az = a.z;
    float2 i_v = __fmul2_rn(f2(h6, h6), f2(a.x, a.y));
    float i_vz = h6 * a.z;
    auto add = [&](float hc) {
        i_v = __ffma2_rn(f2(hc, hc), f2(a.x, a.y), i_v);
        i_vz = fmaf(hc, a.z, i_vz);
    };
    a = accel(M, st.q1, Fm);
    add(h3);
    ax += a.x; ay += a.y; az += a.z;
    a = accel(M, st.q2, Fm);
    add(h3);
    ax += a.x; ay += a.y; az += a.z;
    a = accel(M, st.q3, Fm);
    add(h6);
    const float ipx = fmaf(h, x.vx, hh6 * ax);
    const float ipy = fmaf(h, x.vy, hh6 * ay);
    const float ipz = fmaf(h, x.vz, hh6 * az);
    comp_add2(x.px, x.py, c.px, c.py, ipx, ipy);
    comp_add2(x.vx, x.vy, c.vx, c.vy, i_v.x, i_v.y);
    comp_add2(x.pz, x.vz, c.pz, c.vz, ipz, i_vz);
}

// One whole RK4 step: the operations of rk4_att and rk4_trans, with each
// stage's acceleration formed as soon as its attitude is (fewer values live
// at once).
__device__ __forceinline__ void rk4(const DevModel& M, State& x, Comp& c, float Fm, float tJx, float tJy, float tJz,
                                    float h) {
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f), hh6 = h * h6;
    const Att x0 = {x.qw, x.qx, x.qy, x.qz, x.wx, x.wy, x.wz};
    Att k = att_deriv(M, x0, tJx, tJy, tJz);
    float2 i_q0 = __fmul2_rn(f2(h6, h6), f2(k.qw, k.qx)), i_q1 = __fmul2_rn(f2(h6, h6), f2(k.qy, k.qz));
    float2 i_w = __fmul2_rn(f2(h6, h6), f2(k.wx, k.wy));
    float i_wz = h6 * k.wz;
    const float2 x_q0 = f2(x0.qw, x0.qx), x_q1 = f2(x0.qy, x0.qz), x_w = f2(x0.wx, x0.wy);
    float3 a = accel(M, make_float4(x0.qw, x0.qx, x0.qy, x0.qz), Fm);
    float ax = a.x, ay = a.y, az = a.z;
    float2 i_v = __fmul2_rn(f2(h6, h6), f2(a.x, a.y));
    float i_vz = h6 * a.z;
    Att xs;
    auto stage = [&](float hs) {  // xs = x + hs k; returns the stage attitude
        const float2 H = f2(hs, hs);
        const float2 q0 = __ffma2_rn(H, f2(k.qw, k.qx), x_q0), q1 = __ffma2_rn(H, f2(k.qy, k.qz), x_q1);
        const float2 w = __ffma2_rn(H, f2(k.wx, k.wy), x_w);
        xs.qw = q0.x; xs.qx = q0.y; xs.qy = q1.x; xs.qz = q1.y;
        xs.wx = w.x; xs.wy = w.y; xs.wz = fmaf(hs, k.wz, x0.wz);
        return make_float4(xs.qw, xs.qx, xs.qy, xs.qz);
    };
    auto add = [&](float hc) {
        const float2 H = f2(hc, hc);
        i_q0 = __ffma2_rn(H, f2(k.qw, k.qx), i_q0);
        i_q1 = __ffma2_rn(H, f2(k.qy, k.qz), i_q1);
        i_w = __ffma2_rn(H, f2(k.wx, k.wy), i_w);
        i_wz = fmaf(hc, k.wz, i_wz);
    };
    auto add_v = [&](float hc) {
        i_v = __ffma2_rn(f2(hc, hc), f2(a.x, a.y), i_v);
        i_vz = fmaf(hc, a.z, i_vz);
    };
    a = accel(M, stage(h2), Fm);
    add_v(h3);
    ax += a.x; ay += a.y; az += a.z;
    k = att_deriv(M, xs, tJx, tJy, tJz);
    add(h3);
    a = accel(M, stage(h2), Fm);
    add_v(h3);
    ax += a.x; ay += a.y; az += a.z;
    k = att_deriv(M, xs, tJx, tJy, tJz);
    add(h3);
    a = accel(M, stage(h), Fm);
    add_v(h6);
    k = att_deriv(M, xs, tJx, tJy, tJz);
    add(h6);
    const float ipx = fmaf(h, x.vx, hh6 * ax);
    const float ipy = fmaf(h, x.vy, hh6 * ay);
    const float ipz = fmaf(h, x.vz, hh6 * az);
    comp_add2(x.px, x.py, c.px, c.py, ipx, ipy);
    comp_add2(x.vx, x.vy, c.vx, c.vy, i_v.x, i_v.y);
    comp_add2(x.pz, x.vz, c.pz, c.vz, ipz, i_vz);
    float2 q0 = __fadd2_rn(x_q0, i_q0);
    float2 q1 = __fadd2_rn(x_q1, i_q1);
    const float2 w = __fadd2_rn(x_w, i_w);
    x.wx = w.x; x.wy = w.y; x.wz += i_wz;
    const float2 n2 = __ffma2_rn(q1, q1, __fmul2_rn(q0, q0));
    const float n = rsqrtf(n2.x + n2.y);
    q0 = __fmul2_rn(q0, f2(n, n));
    q1 = __fmul2_rn(q1, f2(n, n));
    x.qw = q0.x; x.qx = q0.y; x.qy = q1.x; x.qz = q1.y;
}

// Uncompensated step (single use: prediction, plant step).
__device__ __forceinline__ void rk4(const DevModel& M, State& x, float Fm, float tJx, float tJy, float tJz, float h) {
    Comp c = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    rk4(M, x, c, Fm, tJx, tJy, tJz, h);
}

__device__ __forceinline__ float4 clamp_input(const DevModel& M, float4 u) {
    u.x = fminf(fmaxf(u.x, M.F_min), M.F_max);
    u.y = fminf(fmaxf(u.y, -M.w_max[0]), M.w_max[0]);
    u.z = fminf(fmaxf(u.z, -M.w_max[1]), M.w_max[1]);
    u.w = fminf(fmaxf(u.w, -M.w_max[2]), M.w_max[2]);
    return u;
}

struct Feasible {
    float F, tx, ty, tz;     // clipped collective thrust and torques
    float gx, gy, gz;        // omega x J omega at the step's start
    float Fm, tJx, tJy, tJz; // F / m and the torques over the inertia (what the dynamics use)
};

// Constraint pipeline of Sec. III-B: desired rate change over dt ->
// desired torque -> rotor thrusts (Gamma^-1) -> clip -> Gamma.  Gamma's
// rows are orthogonal with entries +-1, +-a, +-c, so Gamma^-1 applies as
// T_i = F/4 +- tau_x/(4a) +- tau_y/(4a) +- tau_z/(4c) and Gamma as sums and
// differences of the clipped thrusts.
__device__ __forceinline__ Feasible feasible(const DevModel& M, const State& s, float4 u, float inv_dt) {
    Feasible o;
    o.gx = M.dJx * s.wy * s.wz;
    o.gy = M.dJy * s.wz * s.wx;
    o.gz = M.dJz * s.wx * s.wy;
    const float rx = (u.y - s.wx) * inv_dt, ry = (u.z - s.wy) * inv_dt, rz = (u.w - s.wz) * inv_dt;
    if (M.motor_clip) {
        const float tx = fmaf(M.Jx, rx, o.gx), ty = fmaf(M.Jy, ry, o.gy), tz = fmaf(M.Jz, rz, o.gz);
        const float f0 = 0.25f * u.x, ex = tx * M.q_a, ey = ty * M.q_a, ez = tz * M.q_c;
        const float A = f0 - ez, B = f0 + ez, P = ex + ey, Q = ex - ey;
        const float T0 = fminf(fmaxf(A - P, M.T_min), M.T_max);
        const float T1 = fminf(fmaxf(A + P, M.T_min), M.T_max);
        const float T2 = fminf(fmaxf(B + Q, M.T_min), M.T_max);
        const float T3 = fminf(fmaxf(B - Q, M.T_min), M.T_max);
        const float s01 = T0 + T1, s23 = T2 + T3;
        const float dx = (T1 + T2) - (T0 + T3), dy = (T1 + T3) - (T0 + T2), dz = s23 - s01;
        o.F = s01 + s23;
        o.tx = M.a * dx;
        o.ty = M.a * dy;
        o.tz = M.c_tf * dz;
        o.Fm = o.F * M.inv_mass;
        o.tJx = M.a_Jx * dx;
        o.tJy = M.a_Jy * dy;
        o.tJz = M.c_Jz * dz;
    } else {
        o.F = u.x;
        o.tx = fmaf(M.Jx, rx, o.gx);
        o.ty = fmaf(M.Jy, ry, o.gy);
        o.tz = fmaf(M.Jz, rz, o.gz);
        o.Fm = u.x * M.inv_mass;
        o.tJx = fmaf(M.kx, s.wy * s.wz, rx);
        o.tJy = fmaf(M.ky, s.wz * s.wx, ry);
        o.tJz = fmaf(M.kz, s.wx * s.wy, rz);
    }
    return o;
}

// ------------------------------------------------------------------- cost

// Input and input-change cost of one step (Eq. cost): ||u_j||^2_R and, from
// the second step on, ||u_j - u_{j-1}||^2_{R_Delta}.
__device__ __forceinline__ float input_cost(const DevCost& C, const float4 u, const float4 u_prev, bool rate) {
    const float2 a = f2(u.x, u.y), b = f2(u.z, u.w);
    const float2 t = __ffma2_rn(f2(C.R[2], C.R[3]), __fmul2_rn(b, b), __fmul2_rn(f2(C.R[0], C.R[1]), __fmul2_rn(a, a)));
    float c = t.x + t.y;
    if (rate) {
        const float2 ea = sub2(a, f2(u_prev.x, u_prev.y)), eb = sub2(b, f2(u_prev.z, u_prev.w));
        const float2 r = __ffma2_rn(f2(C.Rd[2], C.Rd[3]), __fmul2_rn(eb, eb),
                                    __fmul2_rn(f2(C.Rd[0], C.Rd[1]), __fmul2_rn(ea, ea)));
        c += r.x + r.y;
    }
    return c;
}

// rho_ref of Sec. IV-C against one reference row staged as four float4:
// (px, py, vx, vy), (pz, vz, wx, wy), (qw, qx, qy, qz), (wz, -, -, -), so
// that the differences pair up for packed arithmetic.  The compensation
// terms c hold minus the low-order parts of p and v.
__device__ __forceinline__ float tracking_cost(const DevCost& C, const State& x, const Comp& c, const float4* row) {
    const float4 r0 = row[0], r1 = row[1], r2 = row[2], r3 = row[3];
    const float2 dp = sub2(sub2(f2(x.px, x.py), f2(r0.x, r0.y)), f2(c.px, c.py));
    const float2 dv = sub2(sub2(f2(x.vx, x.vy), f2(r0.z, r0.w)), f2(c.vx, c.vy));
    const float2 dz = sub2(sub2(f2(x.pz, x.vz), f2(r1.x, r1.y)), f2(c.pz, c.vz));  // (p_z, v_z)
    const float2 dw = sub2(f2(x.wx, x.wy), f2(r1.z, r1.w));
    const float dwz = x.wz - r3.x;
    const float2 qd = __ffma2_rn(f2(x.qy, x.qz), f2(r2.z, r2.w), __fmul2_rn(f2(x.qw, x.qx), f2(r2.x, r2.y)));
    const float dot = qd.x + qd.y;
    float d;
    if (C.quat_metric == 0) {
        d = 1.0f - dot * dot;
    } else {
        d = acosf(fminf(fmaxf(2.0f * dot * dot - 1.0f, -1.0f), 1.0f));
    }
    const float2 sp = __fmul2_rn(dp, dp), sv = __fmul2_rn(dv, dv), sz = __fmul2_rn(dz, dz), sw = __fmul2_rn(dw, dw);
    const float ep = (sp.x + sp.y) + sz.x;
    const float ev = (sv.x + sv.y) + sz.y;
    const float ew = fmaf(dwz, dwz, sw.x + sw.y);
    return fmaf(C.c_p, ep, fmaf(C.c_q, d * d, fmaf(C.c_v, ev, C.c_w * ew)));
}

// Order-preserving map of finite floats to unsigned keys (and back), so
// that the warp's bounding box comes from hardware integer reductions.
__device__ __forceinline__ unsigned float_key(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_float(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A warp's kept-obstacle list, kept across steps: exact for every position
// inside the box [l, h] (the warp's box enlarged by a margin when it was
// built), so it is reused while all of the warp's positions stay inside.
// Replicated in every lane.  n = -1: no list yet; -2: a list did not fit
// (more than 64 kept), lists are not used for the rest of the rollout.
struct WarpList {
    float lx, ly, lz, hx, hy, hz;
    int n;
};

// A warp's kept-obstacle list in shared memory, in pairs: obstacles 2p and
// 2p + 1 are the three float4 at 3p: (x0, x1, y0, y1), (-w0 z0, -w1 z1, w0,
// w1) with w = 1 for a sphere and 0 for a vertical cylinder (whose z does
// not count: w p_z - w z = 0), (-rr0, -rr1, -, -) minus the squared reach
// (radius + r_uav)^2, so that the squared gap is three packed FMAs on -rr.
// Two obstacles are scored with one set of packed FP32x2 instructions.  A
// list of odd length ends with a far-away entry whose squared gap overflows
// to +inf (its term is below the floor: never added; never in collision).
constexpr int kListPairs = 32;          // 64 obstacles per warp
constexpr int kListF4PerWarp = 3 * kListPairs;
constexpr float kFarObstacle = 1.0e30f;

__device__ __forceinline__ void list_put(float4* wob, int idx, const float4 ob) {
    float* f = reinterpret_cast<float*>(wob + 3 * (idx >> 1));
    const int e = idx & 1;
    const bool sph = ob.w >= 0.0f;
    f[e] = ob.x;
    f[2 + e] = ob.y;
    f[4 + e] = sph ? -ob.z : 0.0f;
    f[6 + e] = sph ? 1.0f : 0.0f;
    f[8 + e] = -fabsf(ob.w);
}

// Obstacle term of Sec. IV-D at NP positions p[i] (origin-shifted) of the
// lane's sample: bar_out[i] = the barrier sum c_bar sum_o exp(-beta
// max(gap_o, 0)), each term below its floor 2^-kBarrierFloorLog2 taken as 0,
// and hit_out[i] = whether p[i] is inside an obstacle (the indicator is one
// per state; the caller keeps the count as an exact integer).  NP = 2 scores
// two states of a rollout against one pass over the list: the same terms in
// the same order as two single calls, with twice the independent work per
// loaded obstacle.
//
// Exact culling: the warp's positions are bounded by a box (redux.sync
// min/max on order-preserving keys); each lane tests obstacles of a
// 32-obstacle chunk against the box, and an obstacle is skipped by the whole
// warp when, for every position in the box, its squared gap exceeds the
// cut-off beyond which the term is below its floor (and so it cannot be in
// collision either).  The kept obstacles are copied, in ascending order,
// into the warp's list (WarpList above), built for the box grown by
// `margin` and reused while the positions stay inside; obstacles kept only
// by the margin add exactly +0, so the sum equals the uncut sum.
// With LANES lanes per sample the lanes of a sample take every LANES-th
// pair of kept obstacles and combine by xor-shuffles (bitwise identical
// results on all lanes of the sample).  `reuse` false (launches that count
// evaluated pairs) culls every step.
template <int LANES, int NP>
__device__ __forceinline__ void obstacle_cost_n(const DevCost& C, const float (&px)[NP], const float (&py)[NP],
                                                const float (&pz)[NP], const float4* so, int M, int lane, int wlane,
                                                float4* wob, WarpList& wl, float margin, bool reuse,
                                                float (&bar_out)[NP], bool (&hit_out)[NP], unsigned* kept_out) {
    float bar[NP], smin[NP];  // smin: smallest squared gap (the state is in collision iff <= 0)
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        bar[i] = 0.0f;
        smin[i] = INFINITY;
    }
    if (M > 0) {
        float2 PX[NP], PY[NP], PZ[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            PX[i] = f2(px[i], px[i]);
            PY[i] = f2(py[i], py[i]);
            PZ[i] = f2(pz[i], pz[i]);
        }
        const float2 NB = f2(-C.beta_log2e, -C.beta_log2e);
        // term2: the exponents -beta log2(e) max(gap, 0) of the pair at list
        // position 3q for position i; add: their barrier terms in list
        // order, exactly 0 below the floor whichever box kept the obstacle,
        // so the sum does not depend on the culling.
        auto term2 = [&](const int q, const int i) {
            const float4 A = wob[q], B = wob[q + 1], R = wob[q + 2];
            const float2 dx = sub2(PX[i], f2(A.x, A.y)), dy = sub2(PY[i], f2(A.z, A.w));
            const float2 dz = __ffma2_rn(PZ[i], f2(B.z, B.w), f2(B.x, B.y));  // p_z - z, or 0 (cylinder)
            float2 sg = __ffma2_rn(dx, dx, f2(R.x, R.y));
            sg = __ffma2_rn(dy, dy, sg);
            sg = __ffma2_rn(dz, dz, sg);
            smin[i] = fminf(smin[i], fminf(sg.x, sg.y));
            return __fmul2_rn(NB, f2(fmaxf(sg.x, 0.0f), fmaxf(sg.y, 0.0f)));
        };
        auto add = [&](const float2 a, const int i) {
            if (a.x >= -kBarrierFloorLog2) bar[i] += ex2_ftz(a.x);
            if (a.y >= -kBarrierFloorLog2) bar[i] += ex2_ftz(a.y);
        };
        // Four pairs at a time (one position; two positions: two pairs
        // each): their loads and arithmetic are independent, only the
        // additions stay in list order.
        auto score = [&](int cnt) {
            const int np = (cnt + 1) >> 1;
            int c = lane;
            if (NP == 1) {
                for (; c + 3 * LANES < np; c += 4 * LANES) {
                    const float2 a0 = term2(3 * c, 0), a1 = term2(3 * (c + LANES), 0);
                    const float2 a2 = term2(3 * (c + 2 * LANES), 0), a3 = term2(3 * (c + 3 * LANES), 0);
                    add(a0, 0);
                    add(a1, 0);
                    add(a2, 0);
                    add(a3, 0);
                }
            }
            for (; c + LANES < np; c += 2 * LANES) {
                float2 a[NP][2];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    a[i][0] = term2(3 * c, i);
                    a[i][1] = term2(3 * (c + LANES), i);
                }
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    add(a[i][0], i);
                    add(a[i][1], i);
                }
            }
            for (; c < np; c += LANES) {
#pragma unroll
                for (int i = 0; i < NP; ++i) add(term2(3 * c, i), i);
            }
        };
        // Ends a list of odd length with the far-away entry.
        auto seal = [&](int cnt) {
            if ((cnt & 1) && wlane == 0) list_put(wob, cnt, make_float4(kFarObstacle, 0.0f, 0.0f, 0.0f));
            __syncwarp();
        };
        bool have = false;
        if (reuse && wl.n >= 0) {
            bool in = true;
#pragma unroll
            for (int i = 0; i < NP; ++i)
                in = in && px[i] >= wl.lx && px[i] <= wl.hx && py[i] >= wl.ly && py[i] <= wl.hy && pz[i] >= wl.lz &&
                     pz[i] <= wl.hz;
            have = __all_sync(0xffffffffu, in);
        }
        if (!have) {
            unsigned kxl = float_key(px[0]), kyl = float_key(py[0]), kzl = float_key(pz[0]);
            unsigned kxh = kxl, kyh = kyl, kzh = kzl;
#pragma unroll
            for (int i = 1; i < NP; ++i) {
                const unsigned kx = float_key(px[i]), ky = float_key(py[i]), kz = float_key(pz[i]);
                kxl = min(kxl, kx); kyl = min(kyl, ky); kzl = min(kzl, kz);
                kxh = max(kxh, kx); kyh = max(kyh, ky); kzh = max(kzh, kz);
            }
            const float lox = key_float(__reduce_min_sync(0xffffffffu, kxl));
            const float hix = key_float(__reduce_max_sync(0xffffffffu, kxh));
            const float loy = key_float(__reduce_min_sync(0xffffffffu, kyl));
            const float hiy = key_float(__reduce_max_sync(0xffffffffu, kyh));
            const float loz = key_float(__reduce_min_sync(0xffffffffu, kzl));
            const float hiz = key_float(__reduce_max_sync(0xffffffffu, kzh));
            // Test box: the warp's box, enlarged by the margin while a list
            // is being built.
            const bool build = wl.n != -2;
            float tlx = lox, tly = loy, tlz = loz, thx = hix, thy = hiy, thz = hiz;
            if (build) {
                tlx -= margin; tly -= margin; tlz -= margin;
                thx += margin; thy += margin; thz += margin;
            }
            auto keep_test = [&](int o, const float4 ob) -> bool {
                if (o >= M) return false;
                const float ex = fmaxf(fmaxf(tlx - ob.x, ob.x - thx), 0.0f);
                const float ey = fmaxf(fmaxf(tly - ob.y, ob.y - thy), 0.0f);
                const float ez = ob.w >= 0.0f ? fmaxf(fmaxf(tlz - ob.z, ob.z - thz), 0.0f) : 0.0f;
                const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                return d2 <= (fabsf(ob.w) + C.cull) * 1.0001f;
            };
            // Two 32-obstacle chunks are tested at once; kept obstacles are
            // copied to the warp's list in ascending order.  Building a
            // list appends all chunks; otherwise each chunk is scored as
            // soon as it is compacted.
            const unsigned lt = (1u << wlane) - 1u;
            int base = 0;
            bool fits = build;
            for (int o0 = 0; o0 < M; o0 += 64) {
                const float4 ob0 = o0 + wlane < M ? so[o0 + wlane] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 ob1 = o0 + 32 + wlane < M ? so[o0 + 32 + wlane] : make_float4(0.f, 0.f, 0.f, 0.f);
                const bool k0 = keep_test(o0 + wlane, ob0);
                const bool k1 = keep_test(o0 + 32 + wlane, ob1);
                const unsigned m0 = __ballot_sync(0xffffffffu, k0);
                const unsigned m1 = __ballot_sync(0xffffffffu, k1);
                const int n0 = __popc(m0);
                const int cnt = n0 + __popc(m1);
                if (fits && base + cnt > 2 * kListPairs) {
                    // Too many for one list: score this step chunk by chunk
                    // with the warp's own box, and stop building lists.
                    fits = false;
                    wl.n = -2;
                    tlx = lox; tly = loy; tlz = loz; thx = hix; thy = hiy; thz = hiz;
                    o0 = -64;
                    __syncwarp();
                    continue;
                }
                const int at = fits ? base : 0;
                if (k0) list_put(wob, at + __popc(m0 & lt), ob0);
                if (k1) list_put(wob, at + n0 + __popc(m1 & lt), ob1);
                __syncwarp();
                if (fits) {
                    base += cnt;
                } else {
                    *kept_out += (unsigned)(NP * cnt);
                    seal(cnt);
                    score(cnt);
                    __syncwarp();
                }
            }
            if (fits) {
                wl.lx = tlx; wl.ly = tly; wl.lz = tlz;
                wl.hx = thx; wl.hy = thy; wl.hz = thz;
                wl.n = base;
                seal(base);
                have = true;
            }
        }
        if (have) {
            *kept_out += (unsigned)(NP * wl.n);
            score(wl.n);
            __syncwarp();
        }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        bool hit = smin[i] <= 0.0f;
        if (LANES > 1) {
            unsigned h = hit ? 1u : 0u;
#pragma unroll
            for (int off = LANES / 2; off > 0; off >>= 1) {
                bar[i] += __shfl_xor_sync(0xffffffffu, bar[i], off, LANES);
                h |= __shfl_xor_sync(0xffffffffu, h, off, LANES);
            }
            hit = h != 0u;
        }
        hit_out[i] = hit;
        bar_out[i] = C.c_bar * bar[i];
    }
}

// One position (see obstacle_cost_n).
template <int LANES>
__device__ __forceinline__ float obstacle_cost(const DevCost& C, float px, float py, float pz, const float4* so,
                                               int M, int lane, int wlane, float4* wob, WarpList& wl,
                                               float margin, bool reuse, bool* hit_out, unsigned* kept_out) {
    const float x[1] = {px}, y[1] = {py}, z[1] = {pz};
    float b[1];
    bool h[1];
    obstacle_cost_n<LANES, 1>(C, x, y, z, so, M, lane, wlane, wob, wl, margin, reuse, b, h, kept_out);
    *hit_out = h[0];
    return b[0];
}

// Grid-based collision module: is world position (wx, wy, wz) inside an
// occupied voxel?  Outside the grid is free.
__device__ __forceinline__ bool grid_hit(const DevCost& C, float wx, float wy, float wz) {
    const int ix = (int)floorf((wx - C.g_origin[0]) * C.g_inv_voxel);
    const int iy = (int)floorf((wy - C.g_origin[1]) * C.g_inv_voxel);
    const int iz = (int)floorf((wz - C.g_origin[2]) * C.g_inv_voxel);
    if ((unsigned)ix >= (unsigned)C.gx || (unsigned)iy >= (unsigned)C.gy || (unsigned)iz >= (unsigned)C.gz)
        return false;
    return __ldg(C.grid + ((size_t)iz * C.gy + iy) * C.gx + ix) != 0;
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// ------------------------------------------------- two samples per thread

// The one-sample functions above with every per-sample quantity a float2
// (sample A in .x, sample B in .y) and every operation the same one per
// sample: additions, multiplications and FMAs packed across the two samples
// (FP32x2), minima, maxima, compares and special functions per sample.  The
// packed arithmetic halves the instruction count of the dynamics and the
// cost.  Each sample's results equal the one-sample form's to FP32 rounding,
// not bitwise: the assembler fuses some packed multiply-add pairs that the
// one-sample code rounds separately.
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 clamp2(float2 v, float lo, float hi) {
    return make_float2(fminf(fmaxf(v.x, lo), hi), fminf(fmaxf(v.y, lo), hi));
}

struct State2 {
    float2 px, py, pz, qw, qx, qy, qz, vx, vy, vz, wx, wy, wz;
};
struct Comp2 {
    float2 px, py, pz, vx, vy, vz;
};
struct U2 {  // control (F, omega_x, omega_y, omega_z) of the two samples
    float2 F, wx, wy, wz;
};

__device__ __forceinline__ U2 clamp_input_x2(const DevModel& M, U2 u) {
    u.F = clamp2(u.F, M.F_min, M.F_max);
    u.wx = clamp2(u.wx, -M.w_max[0], M.w_max[0]);
    u.wy = clamp2(u.wy, -M.w_max[1], M.w_max[1]);
    u.wz = clamp2(u.wz, -M.w_max[2], M.w_max[2]);
    return u;
}

__device__ __forceinline__ float2 input_cost_x2(const DevCost& C, const U2& u, const U2& up, bool rate) {
    const float2 tx = fma2(bc(C.R[2]), mul2(u.wy, u.wy), mul2(bc(C.R[0]), mul2(u.F, u.F)));
    const float2 ty = fma2(bc(C.R[3]), mul2(u.wz, u.wz), mul2(bc(C.R[1]), mul2(u.wx, u.wx)));
    float2 c = add2(tx, ty);
    if (rate) {
        const float2 e0 = sub2(u.F, up.F), e1 = sub2(u.wx, up.wx), e2 = sub2(u.wy, up.wy), e3 = sub2(u.wz, up.wz);
        const float2 rx = fma2(bc(C.Rd[2]), mul2(e2, e2), mul2(bc(C.Rd[0]), mul2(e0, e0)));
        const float2 ry = fma2(bc(C.Rd[3]), mul2(e3, e3), mul2(bc(C.Rd[1]), mul2(e1, e1)));
        c = add2(c, add2(rx, ry));
    }
    return c;
}

struct Feasible2 {
    float2 Fm, tJx, tJy, tJz;
};

__device__ __forceinline__ Feasible2 feasible_x2(const DevModel& M, const State2& s, const U2& u, float inv_dt) {
    Feasible2 o;
    const float2 gx = mul2(mul2(bc(M.dJx), s.wy), s.wz);
    const float2 gy = mul2(mul2(bc(M.dJy), s.wz), s.wx);
    const float2 gz = mul2(mul2(bc(M.dJz), s.wx), s.wy);
    const float2 rx = mul2(sub2(u.wx, s.wx), bc(inv_dt));
    const float2 ry = mul2(sub2(u.wy, s.wy), bc(inv_dt));
    const float2 rz = mul2(sub2(u.wz, s.wz), bc(inv_dt));
    if (M.motor_clip) {
        const float2 tx = fma2(bc(M.Jx), rx, gx), ty = fma2(bc(M.Jy), ry, gy), tz = fma2(bc(M.Jz), rz, gz);
        const float2 f0 = mul2(bc(0.25f), u.F);
        const float2 ex = mul2(tx, bc(M.q_a)), ey = mul2(ty, bc(M.q_a)), ez = mul2(tz, bc(M.q_c));
        const float2 A = sub2(f0, ez), B = add2(f0, ez), P = add2(ex, ey), Q = sub2(ex, ey);
        const float2 T0 = clamp2(sub2(A, P), M.T_min, M.T_max);
        const float2 T1 = clamp2(add2(A, P), M.T_min, M.T_max);
        const float2 T2 = clamp2(add2(B, Q), M.T_min, M.T_max);
        const float2 T3 = clamp2(sub2(B, Q), M.T_min, M.T_max);
        const float2 s01 = add2(T0, T1), s23 = add2(T2, T3);
        const float2 dx = sub2(add2(T1, T2), add2(T0, T3));
        const float2 dy = sub2(add2(T1, T3), add2(T0, T2));
        const float2 dz = sub2(s23, s01);
        o.Fm = mul2(add2(s01, s23), bc(M.inv_mass));
        o.tJx = mul2(bc(M.a_Jx), dx);
        o.tJy = mul2(bc(M.a_Jy), dy);
        o.tJz = mul2(bc(M.c_Jz), dz);
    } else {
        o.Fm = mul2(u.F, bc(M.inv_mass));
        o.tJx = fma2(bc(M.kx), mul2(s.wy, s.wz), rx);
        o.tJy = fma2(bc(M.ky), mul2(s.wz, s.wx), ry);
        o.tJz = fma2(bc(M.kz), mul2(s.wx, s.wy), rz);
    }
    return o;
}

struct Att2 {
    float2 qw, qx, qy, qz, wx, wy, wz;
};

// att_deriv with -q_i h_j written as q_i (-h_j) and -(k w_i) w_j as
// (-k w_i) w_j: the same products, so the same roundings.
__device__ __forceinline__ Att2 att_deriv_x2(const DevModel& M, const Att2& s, const Feasible2& f) {
    Att2 d;
    const float2 hx = mul2(bc(0.5f), s.wx), hy = mul2(bc(0.5f), s.wy), hz = mul2(bc(0.5f), s.wz);
    const float2 nx = mul2(bc(-0.5f), s.wx), ny = mul2(bc(-0.5f), s.wy), nz = mul2(bc(-0.5f), s.wz);
    d.qw = fma2(s.qz, nz, fma2(s.qy, ny, mul2(s.qx, nx)));
    d.qx = fma2(s.qz, ny, fma2(s.qy, hz, mul2(s.qw, hx)));
    d.qy = fma2(s.qz, hx, fma2(s.qx, nz, mul2(s.qw, hy)));
    d.qz = fma2(s.qy, nx, fma2(s.qx, hy, mul2(s.qw, hz)));
    d.wx = fma2(mul2(bc(-M.kx), s.wy), s.wz, f.tJx);
    d.wy = fma2(mul2(bc(-M.ky), s.wz), s.wx, f.tJy);
    d.wz = fma2(mul2(bc(-M.kz), s.wx), s.wy, f.tJz);
    return d;
}

struct Q2 {
    float2 qw, qx, qy, qz;
};

__device__ __forceinline__ void accel_x2(const DevModel& M, const Q2& q, float2 Fm, float2& ax, float2& ay,
                                         float2& az) {
    const float2 F2 = mul2(bc(2.0f), Fm);
    ax = mul2(fma2(q.qx, q.qz, mul2(q.qw, q.qy)), F2);
    ay = mul2(fma2(q.qy, q.qz, mul2(mul2(q.qw, q.qx), bc(-1.0f))), F2);
    az = fma2(mul2(bc(-2.0f), Fm), fma2(q.qx, q.qx, mul2(q.qy, q.qy)), sub2(Fm, bc(M.g)));
}

__device__ __forceinline__ void comp_add_x2(float2& x, float2& c, float2 inc) {
    const float2 y = sub2(inc, c);
    const float2 t = add2(x, y);
    c = sub2(sub2(t, x), y);
    x = t;
}

// rk4 for the two samples (the operations of rk4, each stage's
// acceleration formed as soon as its attitude is).
__device__ __forceinline__ void rk4_x2(const DevModel& M, State2& x, Comp2& c, const Feasible2& f, float h) {
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f), hh6 = h * h6;
    const Att2 x0 = {x.qw, x.qx, x.qy, x.qz, x.wx, x.wy, x.wz};
    Att2 k = att_deriv_x2(M, x0, f);
    const float2 H6 = bc(h6), H3 = bc(h3);
    float2 iqw = mul2(H6, k.qw), iqx = mul2(H6, k.qx), iqy = mul2(H6, k.qy), iqz = mul2(H6, k.qz);
    float2 iwx = mul2(H6, k.wx), iwy = mul2(H6, k.wy), iwz = mul2(H6, k.wz);
    float2 ax, ay, az, bx, by, bz;
    accel_x2(M, Q2{x0.qw, x0.qx, x0.qy, x0.qz}, f.Fm, ax, ay, az);
    float2 ivx = mul2(H6, ax), ivy = mul2(H6, ay), ivz = mul2(H6, az);
    Att2 xs;
    auto stage = [&](float hs) {
        const float2 H = bc(hs);
        xs.qw = fma2(H, k.qw, x0.qw); xs.qx = fma2(H, k.qx, x0.qx);
        xs.qy = fma2(H, k.qy, x0.qy); xs.qz = fma2(H, k.qz, x0.qz);
        xs.wx = fma2(H, k.wx, x0.wx); xs.wy = fma2(H, k.wy, x0.wy); xs.wz = fma2(H, k.wz, x0.wz);
        return Q2{xs.qw, xs.qx, xs.qy, xs.qz};
    };
    auto add = [&](float hc) {
        const float2 H = bc(hc);
        iqw = fma2(H, k.qw, iqw); iqx = fma2(H, k.qx, iqx); iqy = fma2(H, k.qy, iqy); iqz = fma2(H, k.qz, iqz);
        iwx = fma2(H, k.wx, iwx); iwy = fma2(H, k.wy, iwy); iwz = fma2(H, k.wz, iwz);
    };
    auto add_v = [&](float2 H) {
        ivx = fma2(H, bx, ivx); ivy = fma2(H, by, ivy); ivz = fma2(H, bz, ivz);
    };
    accel_x2(M, stage(h2), f.Fm, bx, by, bz);
    add_v(H3);
    ax = add2(ax, bx); ay = add2(ay, by); az = add2(az, bz);
    k = att_deriv_x2(M, xs, f);
    add(h3);
    accel_x2(M, stage(h2), f.Fm, bx, by, bz);
    add_v(H3);
    ax = add2(ax, bx); ay = add2(ay, by); az = add2(az, bz);
    k = att_deriv_x2(M, xs, f);
    add(h3);
    accel_x2(M, stage(h), f.Fm, bx, by, bz);
    add_v(H6);
    k = att_deriv_x2(M, xs, f);
    add(h6);
    const float2 Hh = bc(h), HH6 = bc(hh6);
    const float2 ipx = fma2(Hh, x.vx, mul2(HH6, ax));
    const float2 ipy = fma2(Hh, x.vy, mul2(HH6, ay));
    const float2 ipz = fma2(Hh, x.vz, mul2(HH6, az));
    comp_add_x2(x.px, c.px, ipx);
    comp_add_x2(x.py, c.py, ipy);
    comp_add_x2(x.vx, c.vx, ivx);
    comp_add_x2(x.vy, c.vy, ivy);
    comp_add_x2(x.pz, c.pz, ipz);
    comp_add_x2(x.vz, c.vz, ivz);
    float2 qw = add2(x0.qw, iqw), qx = add2(x0.qx, iqx), qy = add2(x0.qy, iqy), qz = add2(x0.qz, iqz);
    x.wx = add2(x0.wx, iwx);
    x.wy = add2(x0.wy, iwy);
    x.wz = add2(x.wz, iwz);
    const float2 ssum = add2(fma2(qy, qy, mul2(qw, qw)), fma2(qz, qz, mul2(qx, qx)));
    const float2 n = f2(rsqrtf(ssum.x), rsqrtf(ssum.y));
    x.qw = mul2(qw, n); x.qx = mul2(qx, n); x.qy = mul2(qy, n); x.qz = mul2(qz, n);
}

__device__ __forceinline__ float2 tracking_cost_x2(const DevCost& C, const State2& x, const Comp2& c,
                                                   const float4* row) {
    const float4 r0 = row[0], r1 = row[1], r2 = row[2], r3 = row[3];
    const float2 dpx = sub2(sub2(x.px, bc(r0.x)), c.px), dpy = sub2(sub2(x.py, bc(r0.y)), c.py);
    const float2 dvx = sub2(sub2(x.vx, bc(r0.z)), c.vx), dvy = sub2(sub2(x.vy, bc(r0.w)), c.vy);
    const float2 dpz = sub2(sub2(x.pz, bc(r1.x)), c.pz), dvz = sub2(sub2(x.vz, bc(r1.y)), c.vz);
    const float2 dwx = sub2(x.wx, bc(r1.z)), dwy = sub2(x.wy, bc(r1.w)), dwz = sub2(x.wz, bc(r3.x));
    const float2 qdx = fma2(x.qy, bc(r2.z), mul2(x.qw, bc(r2.x)));
    const float2 qdy = fma2(x.qz, bc(r2.w), mul2(x.qx, bc(r2.y)));
    const float2 dot = add2(qdx, qdy);
    float2 d;
    if (C.quat_metric == 0) {
        d = sub2(bc(1.0f), mul2(dot, dot));
    } else {
        const float2 t = fma2(mul2(bc(2.0f), dot), dot, bc(-1.0f));
        d = f2(acosf(fminf(fmaxf(t.x, -1.0f), 1.0f)), acosf(fminf(fmaxf(t.y, -1.0f), 1.0f)));
    }
    const float2 ep = add2(add2(mul2(dpx, dpx), mul2(dpy, dpy)), mul2(dpz, dpz));
    const float2 ev = add2(add2(mul2(dvx, dvx), mul2(dvy, dvy)), mul2(dvz, dvz));
    const float2 ew = fma2(dwz, dwz, add2(mul2(dwx, dwx), mul2(dwy, dwy)));
    return fma2(bc(C.c_p), ep, fma2(bc(C.c_q), mul2(d, d), fma2(bc(C.c_v), ev, mul2(bc(C.c_w), ew))));
}

// Box-Muller of box_muller4 for the two samples' Philox outputs rA, rB,
// the float arithmetic packed across the samples.  Returns minus the
// normals (rad cos, rad sin per pair): perturb_neg_x2 multiplies them by
// -sigma, which rounds exactly as sigma times the normal.
struct Z2 {
    float2 z0, z1, z2, z3;
};

__device__ __forceinline__ float2 neg2log_x2(float2 u) {
    float lx, ly;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lx) : "f"(u.x));
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(ly) : "f"(u.y));
    const float2 far = mul2(bc(-1.3862943611198906f), f2(lx, ly));
    const float2 d = sub2(bc(1.0f), u);
    const float2 near = mul2(d, fma2(d, fma2(d, fma2(d, bc(0.5f), bc(0.66666669f)), bc(1.0f)), bc(2.0f)));
    return f2(d.x <= 0.015625f ? near.x : far.x, d.y <= 0.015625f ? near.y : far.y);
}

__device__ __forceinline__ Z2 box_muller_neg_x2(const uint4 rA, const uint4 rB) {
    auto bits = [](unsigned ra, unsigned rb) {
        return f2(__uint_as_float(0x3f800000u | (ra >> 9)), __uint_as_float(0x3f800000u | (rb >> 9)));
    };
    const float2 off = bc(0.99999994039535522f);
    const float2 u0 = sub2(bits(rA.x, rB.x), off), u1 = sub2(bits(rA.y, rB.y), off);
    const float2 u2 = sub2(bits(rA.z, rB.z), off), u3 = sub2(bits(rA.w, rB.w), off);
    const float2 a01 = neg2log_x2(u0), a23 = neg2log_x2(u2);
    const float2 r01 = mul2(a01, f2(rsqrtf(a01.x), rsqrtf(a01.y)));
    const float2 r23 = mul2(a23, f2(rsqrtf(a23.x), rsqrtf(a23.y)));
    const float2 t1 = fma2(bc(6.2831853071795865f), u1, bc(-3.1415926535897932f));
    const float2 t3 = fma2(bc(6.2831853071795865f), u3, bc(-3.1415926535897932f));
    float2 s1, c1, s3, c3;
    __sincosf(t1.x, &s1.x, &c1.x);
    __sincosf(t1.y, &s1.y, &c1.y);
    __sincosf(t3.x, &s3.x, &c3.x);
    __sincosf(t3.y, &s3.y, &c3.y);
    return Z2{mul2(r01, c1), mul2(r01, s1), mul2(r23, c3), mul2(r23, s3)};
}

// u_nom_j + sigma o z with z = -zn (zn from box_muller_neg_x2).
__device__ __forceinline__ U2 perturb_neg_x2(const float4 un, const Z2& zn, const float* sigma) {
    U2 u;
    u.F = add2(bc(un.x), mul2(bc(-sigma[0]), zn.z0));
    u.wx = add2(bc(un.y), mul2(bc(-sigma[1]), zn.z1));
    u.wy = add2(bc(un.z), mul2(bc(-sigma[2]), zn.z2));
    u.wz = add2(bc(un.w), mul2(bc(-sigma[3]), zn.z3));
    return u;
}

__device__ __forceinline__ void kahan_add_x2(float2& sum, float2& comp, float2 v) {
    const float2 y = sub2(v, comp);
    const float2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// ------------------------------------------------------------ TMA + mbarrier

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Non-blocking test of one phase of the barrier.
__device__ __forceinline__ bool mbar_test_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Default bound of every device-side wait, in polls of the barrier (each
// poll may suspend for a hardware-defined time): about a second.
constexpr long long kWaitPolls = 1ll << 22;

// Bounded wait on one phase of the barrier, then false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, long long polls) {
    for (long long i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Bounded wait that also gives up when another warp of the block has
// flagged an abort; a wait that runs out raises the flag itself, so a
// stuck pipeline drains quickly instead of every later wait timing out.
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned parity, volatile int* abort_flag,
                                                   long long polls) {
    if (mbar_test_wait(bar, parity)) return true;
    for (long long i = 0; i < polls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// ------------------------------------------------------------ block helpers

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// ------------------------------------------------------------ cost pairs

// Weight below which exp(-x) is zero in FP32 (denormals included): such
// samples contribute exactly nothing and are skipped.
constexpr float kMaxExpArg = 104.0f;

// A rollout cost S_k = c_obs (states in collision) + (S - Sc), the
// compensated sum of the continuous terms, is carried as an unevaluated
// pair of floats (hi, lo) with hi + lo equal to it to about 2^-44 relative:
// the product c_obs n by its FMA-exact error, the additions by TwoSum
// (Knuth), and hi the FP32 rounding of the sum (|lo| <= ulp(hi) / 2).  The
// minimum, the differences S_k - rho and the softmin arguments are then
// formed in FP32 arithmetic with a resolution far below the FP32 rounding
// of the cost itself, so the large collision term does not swamp the
// differences the weights depend on; nothing runs on the FP64 pipe, which
// on this GPU issues a small fraction of the FP32 rate.  The intrinsics keep
// the compiler from fusing the product into a later addition.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ float2 cost_pair(float c_obs, int nhit, float S, float Sc) {
    const float n = (float)nhit;  // exact (nhit <= N)
    const float p = __fmul_rn(c_obs, n);
    const float pe = fmaf(c_obs, n, -p);  // c_obs n = p + pe exactly
    const float2 h = two_sum(p, S);       // p + S = h.x + h.y exactly
    return two_sum(h.x, __fadd_rn(h.y, __fsub_rn(pe, Sc)));
}

// Order-preserving 64-bit key of a pair (hi, lo): lexicographic in hi, then
// lo, which orders pairs by value.
__device__ __forceinline__ unsigned long long pair_key(float2 v) {
    return ((unsigned long long)float_key(v.x) << 32) | float_key(v.y);
}

__device__ __forceinline__ float2 key_pair(unsigned long long k) {
    return make_float2(key_float((unsigned)(k >> 32)), key_float((unsigned)k));
}

// Smallest key of the warp, by two 32-bit hardware reductions.
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long k) {
    const unsigned hi = (unsigned)(k >> 32);
    const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? (unsigned)k : 0xffffffffu);
    return ((unsigned long long)mh << 32) | ml;
}

// Softmin weight exp(-(v - rho) / lambda) of a cost pair v >= rho (Eq.
// cost_2 after the minimum shift); exactly 0 for a non-finite cost and below
// the FP32 range.
__device__ __forceinline__ float softmin_weight(float2 v, float2 rho, float lambda) {
    if (!(v.x < INFINITY)) return 0.0f;
    const float dv = __fadd_rn(__fsub_rn(v.x, rho.x), __fsub_rn(v.y, rho.y));
    const float xarg = dv / lambda;
    return xarg <= kMaxExpArg ? expf(-xarg) : 0.0f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Dynamic shared memory layout (byte offsets), identical on host and device.
// The pipelined variant adds, per group of 32 samples, a ring of kRing
// slots (kSlotF4 float4 per lane, stored lane-contiguous: the position and
// the step's tracking cost, the position's compensation terms, and the
// control) from the warp that integrates the position to the cost lanes,
// and kBarsPerSlot mbarriers per slot: [2] / [3] full / empty of that ring,
// [0] / [1] full / empty of the noise ring (one float4 per lane and slot)
// that the noise warp of the PIPE >= 2 forms fills, [4] / [5] full / empty
// of the attitude ring (kAttF4 float4 per lane and slot) from the attitude
// warp to the translation warp of the PIPE == 3 form.
constexpr int kRing = 4;
constexpr int kSlotF4 = 3;
constexpr int kAttF4 = 6;
__host__ __device__ constexpr int bars_per_slot(int pipe) { return pipe == 3 ? 6 : 4; }
// States the cost lanes of the pipelined form score per pass over their
// kept-obstacle list (at most kRing).  Closed-loop step (K=16384, N=100, 64
// spheres), split form: 1, 2, 3, 4 states per pass take 90.3, 76.9, 76.2,
// 75.8 us.
constexpr int kStatesPerPass = 4;

struct SmemLayout {
    unsigned obs, ref, u, S, e, list, part, wlist, xring, nring, qring, bars, total;
};

__host__ __device__ inline unsigned align_up(unsigned v, unsigned a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int N_max, int M_max, int block, int lanes, int pipe, int spt) {
    SmemLayout L;
    const int spb = pipe ? block / (pipe + lanes) : spt * block / lanes;
    const int npart = block > N_max ? block : N_max;
    const unsigned slots = pipe ? (unsigned)(spb / 32) * kRing * 32u : 0u;
    unsigned o = 0;
    L.obs = o;  o = align_up(o + 16u * (unsigned)M_max, 128);
    L.ref = o;  o = align_up(o + 64u * (unsigned)(N_max + 1), 128);
    L.u = o;    o = align_up(o + 16u * (unsigned)N_max, 128);
    L.S = o;    o = align_up(o + 8u * (unsigned)spb, 128);
    L.e = o;    o = align_up(o + 4u * (unsigned)spb, 128);
    L.list = o; o = align_up(o + 4u * (unsigned)spb, 128);
    L.part = o; o = align_up(o + 16u * (unsigned)npart, 128);
    L.wlist = o; o = align_up(o + 48u * (unsigned)block, 128);  // 96 float4 (32 obstacle pairs) per warp
    L.xring = o; o = align_up(o + 16u * kSlotF4 * slots, 128);
    L.nring = o; o = align_up(o + (pipe >= 2 ? 16u * slots : 0u), 128);
    L.qring = o; o = align_up(o + (pipe == 3 ? 16u * kAttF4 * slots : 0u), 128);
    L.bars = o;  o = align_up(o + 8u * (unsigned)bars_per_slot(pipe) * (slots / 32u), 128);
    L.total = o;
    return L;
}

// --------------------------------------------------------------- the kernel

// MINB > 1: an instantiation for blocks of at most 128 threads compiled to
// fit MINB blocks per SM (a register budget of 65536 / (128 MINB) per
// thread), for launches that fill the GPU and are bound by issue rate.
template <int LANES, int PIPE, int MINB, int SPT>
__global__ void __launch_bounds__(MINB > 1 ? 128 : 512, MINB) mppi_step_kernel(const LaunchArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ DevInstance sI;
    __shared__ int s_tile, s_inst, s_tile_in_inst, s_last, s_count, s_abort, s_lost;
    __shared__ float s_x0[16], s_xhat[13];
    __shared__ unsigned long long s_wkey[32];  // per-(virtual) warp minimum cost key
    __shared__ int s_wcnt[32];                 // per-(virtual) warp contributor count
    __shared__ float s_red[32];                // per-(virtual) warp weight sum
    __shared__ uint4 s_rk[5];  // Philox round keys of the tile's instance
    __shared__ uint2 s_pt;     // the first round's per-tile words

    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    // PIPE 1: samples [0, spb) have a dynamics thread (tid < spb) and LANES
    // cost lanes (tid >= spb) in separate warps; PIPE 2: also a noise thread
    // (spb <= tid < 2 spb); PIPE 3: the dynamics split over an attitude
    // thread (tid < spb) and a translation thread (2 spb <= tid < 3 spb),
    // with the noise thread in between; otherwise LANES lanes per sample, or
    // (SPT == 2) two samples per thread, tid and nthreads + tid.
    const int spb = PIPE ? nthreads / (PIPE + LANES) : SPT * nthreads / LANES;
    const int group = PIPE ? (tid < PIPE * spb ? tid % spb : (tid - PIPE * spb) / LANES) : tid / LANES;
    const int lane = PIPE ? (tid < PIPE * spb ? 0 : (tid - PIPE * spb) % LANES) : tid % LANES;
    const int warp = tid >> 5, wlane = tid & 31, nwarps = nthreads >> 5;

    const SmemLayout L = smem_layout(a.N_max, a.M_max, nthreads, LANES, PIPE, SPT);
    float4* sobs = reinterpret_cast<float4*>(smem + L.obs);
    float4* sref = reinterpret_cast<float4*>(smem + L.ref);
    float4* su = reinterpret_cast<float4*>(smem + L.u);
    float2* sS = reinterpret_cast<float2*>(smem + L.S);  // cost pairs (hi, lo)
    float* sE = reinterpret_cast<float*>(smem + L.e);
    int* slist = reinterpret_cast<int*>(smem + L.list);
    float4* spart = reinterpret_cast<float4*>(smem + L.part);
    float4* wob = reinterpret_cast<float4*>(smem + L.wlist) + kListF4PerWarp * (threadIdx.x >> 5);

    const unsigned bar = smem_addr(&mbar);
    unsigned phase = 0;
    if (tid == 0) {
        mbar_init(bar, 1);
        s_abort = 0;
        s_lost = 0;
        if (PIPE)  // per (group, slot): [3] state empty (cost lanes) counts 32 LANES arrivals, the others 32
            for (int b = 0; b < (spb / 32) * kRing * bars_per_slot(PIPE); ++b)
                mbar_init(smem_addr(smem + L.bars) + 8u * b, b % bars_per_slot(PIPE) == 3 ? 32 * LANES : 32);
    }
    __syncthreads();
    unsigned g_run = 0;  // pipeline steps run so far by this block (ring slot / phase)

    const DevModel& Mdl = a.M;
    const DevCost& C = a.C;
    const int n_tiles = a.n_tiles_dev ? *a.n_tiles_dev : a.n_tiles;
    const long long wait_polls = a.wait_polls > 0 ? a.wait_polls : kWaitPolls;
    // Kept-obstacle lists are reused across steps, except in launches that
    // count evaluated pairs: those cull every step with the warp's own box.
    const bool reuse_lists = a.stats == nullptr;
    const float cull_margin = reuse_lists ? C.cull_margin : 0.0f;

    for (int round = 0;; ++round) {
        // ---------------------------------------------------- pick a tile
        if (tid == 0) {
            int t;
            if (a.tile_counter) t = (int)atomicAdd(a.tile_counter, 1u);
            else t = round == 0 ? (int)blockIdx.x : n_tiles;
            s_tile = t;
            if (t < n_tiles) {
                const int2 tm = a.tile_map ? a.tile_map[t] : make_int2(0, t);
                s_inst = tm.x;
                s_tile_in_inst = tm.y;
                sI = a.insts ? a.insts[tm.x] : a.single;
            }
        }
        __syncthreads();
        if (s_tile >= n_tiles) break;
        // A block whose obstacle copy never landed (s_lost) or whose
        // pipeline gave up a wait (s_abort) keeps taking tiles, so that every
        // instance is still merged and given a status, but skips the copy
        // and flags each instance it touches: its outputs are unspecified.
        const bool lost = s_lost != 0;
        const int inst = s_inst;
        const int tile = s_tile_in_inst;
        const int K = sI.K, N = sI.N, M = sI.M;
        const float dt = sI.dt, inv_dt = 1.0f / sI.dt, lambda = sI.lambda;
        const unsigned long long iter = sI.iter_dev ? *sI.iter_dev : sI.iter;
        if (tid < 5) s_rk[tid] = philox_round_keys(sI.key0, sI.key1, (unsigned)tid);
        if (tid == 0) {
            const uint4 rk0 = philox_round_keys(sI.key0, sI.key1, 0u);
            s_pt = philox_pre_tile(iter, &rk0);
        }
        float sigma[4] = {sI.sigma[0], sI.sigma[1], sI.sigma[2], sI.sigma[3]};

        // ---------------------------------- stage inputs in shared memory
        // Obstacles by one bulk TMA copy (overlaps the loads below).
        if (tid == 0 && M > 0 && !lost && !a.stall_obstacle_copy)
            bulk_load(smem_addr(sobs), sI.obs, 16u * (unsigned)M, bar);
        if (tid == 0 && (lost || s_abort)) atomicOr(&a.errflags[inst], ERR_TIMEOUT);
        if (tid < 13) s_xhat[tid] = sI.x_hat[tid];
        // The reference window and the nominal are loaded alongside x_hat
        // (no dependent round trip); the reference positions are shifted
        // once x_hat is in shared memory, each row by the thread that
        // loaded it.
        for (int j = tid; j <= N; j += nthreads) {
            const float* r = sI.ref + 13 * (size_t)j;
            sref[4 * j + 0] = make_float4(r[0], r[1], r[7], r[8]);
            sref[4 * j + 1] = make_float4(r[2], r[9], r[10], r[11]);
            sref[4 * j + 2] = make_float4(r[3], r[4], r[5], r[6]);
            sref[4 * j + 3] = make_float4(r[12], 0.0f, 0.0f, 0.0f);
        }
        for (int j = tid; j < N; j += nthreads) {
            const float* u = sI.u_nom + 4 * (size_t)j;
            su[j] = make_float4(u[0], u[1], u[2], u[3]);
        }
        __syncthreads();
        // Origin shift to the state estimate's position: translation
        // invariant in exact arithmetic, keeps FP32 positions small.
        const float p0x = s_xhat[0], p0y = s_xhat[1], p0z = s_xhat[2];
        for (int j = tid; j <= N; j += nthreads) {
            sref[4 * j + 0].x -= p0x;
            sref[4 * j + 0].y -= p0y;
            sref[4 * j + 1].x -= p0z;
        }
        if (tid == 0) {
            State x;
            x.px = 0.0f; x.py = 0.0f; x.pz = 0.0f;
            x.qw = s_xhat[3]; x.qx = s_xhat[4]; x.qy = s_xhat[5]; x.qz = s_xhat[6];
            x.vx = s_xhat[7]; x.vy = s_xhat[8]; x.vz = s_xhat[9];
            x.wx = s_xhat[10]; x.wy = s_xhat[11]; x.wz = s_xhat[12];
            if (C.delay > 0.0f) {
                // Delay compensation (Sec. IV-E): predict x_hat forward.
                const float* u = sI.u_nom;
                const float4 u0 = clamp_input(Mdl, make_float4(u[0], u[1], u[2], u[3]));
                const Feasible f = feasible(Mdl, x, u0, inv_dt);
                rk4(Mdl, x, f.Fm, f.tJx, f.tJy, f.tJz, C.delay);
            }
            s_x0[0] = x.px; s_x0[1] = x.py; s_x0[2] = x.pz; s_x0[3] = x.qw; s_x0[4] = x.qx;
            s_x0[5] = x.qy; s_x0[6] = x.qz; s_x0[7] = x.vx; s_x0[8] = x.vy; s_x0[9] = x.vz;
            s_x0[10] = x.wx; s_x0[11] = x.wy; s_x0[12] = x.wz;
        }
        if (M > 0) {
            if (!lost) {
                if (!mbar_wait_bounded(bar, phase, wait_polls)) {
                    // The copy did not land in time: flag the instance and
                    // give it one more bounded wait to land before shared
                    // memory is reused; after that the barrier is given up.
                    if (tid == 0) atomicOr(&a.errflags[inst], ERR_TIMEOUT);
                    if (!mbar_wait_bounded(bar, phase, wait_polls)) s_lost = 1;
                }
                phase ^= 1u;
            }
            for (int o = tid; o < M; o += nthreads) {
                const float4 ob = sobs[o];
                const float reach = fabsf(ob.w) + C.r_uav;
                const float rr = reach * reach;
                sobs[o] = ob.w < 0.0f ? make_float4(ob.x - p0x, ob.y - p0y, 0.0f, -rr)
                                      : make_float4(ob.x - p0x, ob.y - p0y, ob.z - p0z, rr);
            }
        }
        __syncthreads();

        // --------------------------------------------------- rollouts
        if constexpr (PIPE == 0 && SPT == 2) {
            // Two samples per thread, A (tile sample tid) and B (nthreads +
            // tid), one thread per sample otherwise: the one-thread form's
            // arithmetic packed across the two, their positions scored in one
            // pass over the warp's kept-obstacle list.
            const int gA = tid, gB = nthreads + tid;
            const int kA_raw = tile * spb + gA, kB_raw = tile * spb + gB;
            const bool validA = kA_raw < K, validB = kB_raw < K;
            const unsigned kA = (unsigned)(validA ? kA_raw : K - 1), kB = (unsigned)(validB ? kB_raw : K - 1);
            State2 x;
            x.px = bc(s_x0[0]); x.py = bc(s_x0[1]); x.pz = bc(s_x0[2]); x.qw = bc(s_x0[3]); x.qx = bc(s_x0[4]);
            x.qy = bc(s_x0[5]); x.qz = bc(s_x0[6]); x.vx = bc(s_x0[7]); x.vy = bc(s_x0[8]); x.vz = bc(s_x0[9]);
            x.wx = bc(s_x0[10]); x.wy = bc(s_x0[11]); x.wz = bc(s_x0[12]);
            Comp2 cmp = {bc(0.f), bc(0.f), bc(0.f), bc(0.f), bc(0.f), bc(0.f)};
            float2 S = bc(0.0f), Sc = bc(0.0f);
            int nhitA = 0, nhitB = 0;
            unsigned kept = 0;  // 2 x obstacles evaluated by this warp per position pair
            WarpList wl;
            wl.n = -1;
            float bars[2];
            bool hits[2];
            auto score = [&](float2 qx, float2 qy, float2 qz) {
                const float px[2] = {qx.x, qx.y}, py[2] = {qy.x, qy.y}, pz[2] = {qz.x, qz.y};
                obstacle_cost_n<1, 2>(C, px, py, pz, sobs, M, lane, wlane, wob, wl, cull_margin, reuse_lists, bars,
                                      hits, &kept);
                if (C.grid) {
                    hits[0] |= grid_hit(C, qx.x + p0x, qy.x + p0y, qz.x + p0z);
                    hits[1] |= grid_hit(C, qx.y + p0x, qy.y + p0y, qz.y + p0z);
                }
                nhitA += hits[0] ? 1 : 0;
                nhitB += hits[1] ? 1 : 0;
                return f2(bars[0], bars[1]);
            };
            {
                const float2 tc = tracking_cost_x2(C, x, cmp, &sref[0]);
                kahan_add_x2(S, Sc, add2(tc, score(x.px, x.py, x.pz)));
            }
            // The previous step's controls and the samples' first-round Philox
            // words live in shared memory, read once per step: in registers they
            // pushed the loop past the 128-register budget into local-memory
            // spills (batched launch 4.56 -> 4.53 ms).
            __shared__ float4 s_up[2 * 128];  // u_{j-1} of samples A and B, per thread (block <= 128)
            __shared__ uint4 s_pp[128];       // PhiloxPre of A and B, per thread
            s_up[2 * tid] = make_float4(0.f, 0.f, 0.f, 0.f);
            s_up[2 * tid + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            {
                const PhiloxPre pa = philox_pre_sample(kA, iter, s_rk), pb = philox_pre_sample(kB, iter, s_rk);
                s_pp[tid] = make_uint4(pa.z, pa.w, pb.z, pb.w);
            }
            for (int j = 0; j < N; ++j) {
                const uint4 pq = s_pp[tid];
                PhiloxPre ppA, ppB;
                ppA.z = pq.x; ppA.w = pq.y; ppB.z = pq.z; ppB.w = pq.w;
                const Z2 zn = box_muller_neg_x2(philox_pre((unsigned)j, ppA, &s_pt, s_rk),
                                                philox_pre((unsigned)j, ppB, &s_pt, s_rk));
                const U2 u = clamp_input_x2(Mdl, perturb_neg_x2(su[j], zn, sigma));
                U2 u_prev;
                {
                    const float4 a = s_up[2 * tid], b = s_up[2 * tid + 1];
                    u_prev.F = f2(a.x, a.y); u_prev.wx = f2(a.z, a.w);
                    u_prev.wy = f2(b.x, b.y); u_prev.wz = f2(b.z, b.w);
                }
                float2 step = input_cost_x2(C, u, u_prev, j > 0);
                s_up[2 * tid] = make_float4(u.F.x, u.F.y, u.wx.x, u.wx.y);
                s_up[2 * tid + 1] = make_float4(u.wy.x, u.wy.y, u.wz.x, u.wz.y);
                const Feasible2 f = feasible_x2(Mdl, x, u, inv_dt);
                rk4_x2(Mdl, x, cmp, f, dt);
                step = add2(step, tracking_cost_x2(C, x, cmp, &sref[4 * (j + 1)]));
                step = add2(step, score(sub2(x.px, cmp.px), sub2(x.py, cmp.py), sub2(x.pz, cmp.pz)));
                kahan_add_x2(S, Sc, step);
            }
            if (a.stats) {
                const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, validA)) +
                                        __popc(__ballot_sync(0xffffffffu, validB));
                if (wlane == 0 && kept) atomicAdd(a.stats, (unsigned long long)(kept / 2) * nvalid);
            }
            const float2 SkA = cost_pair(C.c_obs, nhitA, S.x, Sc.x), SkB = cost_pair(C.c_obs, nhitB, S.y, Sc.y);
            if (validA && sI.costs) sI.costs[kA_raw] = SkA.x;
            if (validB && sI.costs) sI.costs[kB_raw] = SkB.x;
            sS[gA] = (validA && isfinite(SkA.x)) ? SkA : make_float2(INFINITY, 0.0f);
            sS[gB] = (validB && isfinite(SkB.x)) ? SkB : make_float2(INFINITY, 0.0f);
            __syncthreads();
        } else if constexpr (PIPE == 0) {
            const int k_raw = tile * spb + group;
            const bool valid = k_raw < K;
            const unsigned k = (unsigned)(valid ? k_raw : K - 1);
            State x;
            x.px = s_x0[0]; x.py = s_x0[1]; x.pz = s_x0[2]; x.qw = s_x0[3]; x.qx = s_x0[4];
            x.qy = s_x0[5]; x.qz = s_x0[6]; x.vx = s_x0[7]; x.vy = s_x0[8]; x.vz = s_x0[9];
            x.wx = s_x0[10]; x.wy = s_x0[11]; x.wz = s_x0[12];

            // S_k = c_obs * (states in collision) + the continuous cost, kept
            // apart: the indicator is an exact count and the continuous part a
            // compensated FP32 sum, combined into a float pair (cost_pair).
            Comp cmp = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float S = 0.0f, Sc = 0.0f;
            int nhit = 0;
            bool hit = false;
            unsigned kept = 0;  // obstacles evaluated by this warp (uniform over the warp)
            WarpList wl;
            wl.n = -1;
            kahan_add(S, Sc, tracking_cost(C, x, cmp, &sref[0]) +
                                 obstacle_cost<LANES>(C, x.px, x.py, x.pz, sobs, M, lane, wlane, wob, wl, cull_margin,
                                                      reuse_lists, &hit, &kept));
            if (C.grid) hit |= grid_hit(C, x.px + p0x, x.py + p0y, x.pz + p0z);
            nhit += hit ? 1 : 0;
            float4 u_prev = make_float4(0.f, 0.f, 0.f, 0.f);
            const PhiloxPre ppre = philox_pre_sample(k, iter, s_rk);
            for (int j = 0; j < N; ++j) {
                const float4 d = noise_delta(normals4_pre((unsigned)j, ppre, &s_pt, s_rk), sigma);
                const float4 un = su[j];
                const float4 u = clamp_input(Mdl, perturb(un, d));
                float step = input_cost(C, u, u_prev, j > 0);
                u_prev = u;
                const Feasible f = feasible(Mdl, x, u, inv_dt);
                rk4(Mdl, x, cmp, f.Fm, f.tJx, f.tJy, f.tJz, dt);
                step += tracking_cost(C, x, cmp, &sref[4 * (j + 1)]);
                step += obstacle_cost<LANES>(C, x.px - cmp.px, x.py - cmp.py, x.pz - cmp.pz, sobs, M, lane, wlane, wob,
                                             wl, cull_margin, reuse_lists, &hit, &kept);
                if (C.grid) hit |= grid_hit(C, (x.px - cmp.px) + p0x, (x.py - cmp.py) + p0y, (x.pz - cmp.pz) + p0z);
                nhit += hit ? 1 : 0;
                kahan_add(S, Sc, step);
            }
            if (a.stats) {
                // Evaluated pairs: kept obstacles x valid samples of this warp.
                const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, valid && lane == 0));
                if (wlane == 0 && kept) atomicAdd(a.stats, (unsigned long long)kept * nvalid);
            }
            if (lane == 0) {
                const float2 Sk = cost_pair(C.c_obs, nhit, S, Sc);
                if (valid && sI.costs) sI.costs[k_raw] = Sk.x;
                sS[group] = (valid && isfinite(Sk.x)) ? Sk : make_float2(INFINITY, 0.0f);
            }
            __syncthreads();
        } else {
            // Pipelined rollout.  The dynamics thread of a sample draws the
            // noise (one step ahead, overlapping the RK4 chain; with PIPE == 2
            // a noise thread in its own warp draws it and hands it over
            // through a second ring), clamps the control, runs the constraint
            // pipeline and RK4 and forms the step's tracking cost; it hands
            // the new position (with its compensation terms), that cost and
            // the control to the sample's cost lanes through a ring in shared
            // memory.  The cost lanes add the input and input-change cost and
            // score the positions, two states per pass, against the obstacles
            // and the grid while the dynamics thread is already integrating
            // the next steps.  With PIPE == 3 the noise thread also forms the
            // clamped control, and the dynamics are split: the attitude
            // thread runs the constraint pipeline and the attitude part of
            // RK4 and hands the stage attitudes, the new attitude and rates
            // and F/m to the translation thread, which integrates velocity
            // and position, forms the tracking cost and feeds the cost lanes.
            // Every wait is bounded.
            const bool is_cost = tid >= PIPE * spb;
            const bool is_noise = PIPE >= 2 && tid >= spb && tid < 2 * spb;
            const bool is_trans = PIPE == 3 && tid >= 2 * spb && !is_cost;
            const int pw = group >> 5;  // warp pair
            float4* xring = reinterpret_cast<float4*>(smem + L.xring);
            const unsigned bars = smem_addr(smem + L.bars);
            volatile int* abort_flag = &s_abort;
            auto slot_of = [&](unsigned g) { return (int)(g % kRing); };
            auto bar_of = [&](int slot, int kind) {
                return bars + 8u * (unsigned)((pw * kRing + slot) * bars_per_slot(PIPE) + kind);
            };
            // Field f of this lane's entry in a ring slot.
            auto ring_at = [&](int slot, int f) { return xring + ((pw * kRing + slot) * kSlotF4 + f) * 32 + (group & 31); };
            constexpr int X_FULL = 2, X_EMPTY = 3;
            // Noise ring (PIPE == 2): delta for step g in slot g % kRing.
            float4* nring = reinterpret_cast<float4*>(smem + L.nring);
            auto nring_at = [&](int slot) { return nring + (pw * kRing + slot) * 32 + (group & 31); };
            constexpr int N_FULL = 0, N_EMPTY = 1;
            // Attitude ring (PIPE == 3): field f of this lane's entry.
            float4* qring = reinterpret_cast<float4*>(smem + L.qring);
            auto qring_at = [&](int slot, int f) {
                return qring + ((pw * kRing + slot) * kAttF4 + f) * 32 + (group & 31);
            };
            constexpr int Q_FULL = 4, Q_EMPTY = 5;
            const int k_raw = tile * spb + group;
            const bool valid = k_raw < K;
            const unsigned k = (unsigned)(valid ? k_raw : K - 1);
            State x;
            x.px = s_x0[0]; x.py = s_x0[1]; x.pz = s_x0[2]; x.qw = s_x0[3]; x.qx = s_x0[4];
            x.qy = s_x0[5]; x.qz = s_x0[6]; x.vx = s_x0[7]; x.vy = s_x0[8]; x.vz = s_x0[9];
            x.wx = s_x0[10]; x.wy = s_x0[11]; x.wz = s_x0[12];
            Comp cmp = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (is_noise) {
                // Noise thread (PIPE >= 2): draws delta for every step ahead of
                // the dynamics and hands it over through its own ring (PIPE ==
                // 3: the clamped control u_nom_j + delta instead).
                const PhiloxPre ppre = philox_pre_sample(k, iter, s_rk);
                for (int j = 0; j < N; ++j) {
                    const unsigned g = g_run + (unsigned)j;
                    const int slot = slot_of(g);
                    const unsigned ph = (g / kRing) & 1u;
                    float4 d = noise_delta(normals4_pre((unsigned)j, ppre, &s_pt, s_rk), sigma);
                    if (PIPE == 3) d = clamp_input(Mdl, perturb(su[j], d));
                    if (g >= (unsigned)kRing) mbar_wait_or_abort(bar_of(slot, N_EMPTY), ph ^ 1u, abort_flag, wait_polls);
                    *nring_at(slot) = d;
                    mbar_arrive(bar_of(slot, N_FULL));
                }
            } else if (PIPE == 3 && !is_cost && !is_trans) {
                // Attitude thread: control from the noise ring, constraint
                // pipeline, attitude part of RK4.
                for (int j = 0; j < N; ++j) {
                    const unsigned g = g_run + (unsigned)j;
                    const int slot = slot_of(g);
                    const unsigned ph = (g / kRing) & 1u;
                    mbar_wait_or_abort(bar_of(slot, N_FULL), ph, abort_flag, wait_polls);
                    const float4 u = *nring_at(slot);
                    mbar_arrive(bar_of(slot, N_EMPTY));
                    const Feasible f = feasible(Mdl, x, u, inv_dt);
                    const Stages st = rk4_att(Mdl, x, f.tJx, f.tJy, f.tJz, dt);
                    if (g >= (unsigned)kRing) mbar_wait_or_abort(bar_of(slot, Q_EMPTY), ph ^ 1u, abort_flag, wait_polls);
                    *qring_at(slot, 0) = st.q1;
                    *qring_at(slot, 1) = st.q2;
                    *qring_at(slot, 2) = st.q3;
                    *qring_at(slot, 3) = make_float4(x.qw, x.qx, x.qy, x.qz);
                    *qring_at(slot, 4) = make_float4(x.wx, x.wy, x.wz, f.Fm);
                    *qring_at(slot, 5) = u;
                    mbar_arrive(bar_of(slot, Q_FULL));
                }
            } else if (is_trans) {
                // Translation thread: velocity and position from the stage
                // attitudes, the step's input, input-change and tracking cost
                // (in the one-thread form's order), hand-over to the cost lanes.
                float4 u_prev = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int j = 0; j < N; ++j) {
                    const unsigned g = g_run + (unsigned)j;
                    const int slot = slot_of(g);
                    const unsigned ph = (g / kRing) & 1u;
                    mbar_wait_or_abort(bar_of(slot, Q_FULL), ph, abort_flag, wait_polls);
                    Stages st;
                    st.q1 = *qring_at(slot, 0);
                    st.q2 = *qring_at(slot, 1);
                    st.q3 = *qring_at(slot, 2);
                    const float4 qn = *qring_at(slot, 3), wf = *qring_at(slot, 4), u = *qring_at(slot, 5);
                    mbar_arrive(bar_of(slot, Q_EMPTY));
                    rk4_trans(Mdl, x, cmp, make_float4(x.qw, x.qx, x.qy, x.qz), st, wf.w, dt);
                    x.qw = qn.x; x.qx = qn.y; x.qy = qn.z; x.qz = qn.w;
                    x.wx = wf.x; x.wy = wf.y; x.wz = wf.z;
                    float scost = input_cost(C, u, u_prev, j > 0);
                    u_prev = u;
                    scost += tracking_cost(C, x, cmp, &sref[4 * (j + 1)]);
                    if (g >= (unsigned)kRing) mbar_wait_or_abort(bar_of(slot, X_EMPTY), ph ^ 1u, abort_flag, wait_polls);
                    *ring_at(slot, 0) = make_float4(x.px, x.py, x.pz, scost);
                    *ring_at(slot, 1) = make_float4(cmp.px, cmp.py, cmp.pz, 0.0f);
                    mbar_arrive(bar_of(slot, X_FULL));
                }
            } else if (!is_cost) {
                const PhiloxPre ppre = philox_pre_sample(k, iter, s_rk);
                float4 d_next = make_float4(0.f, 0.f, 0.f, 0.f);
                if (PIPE == 1) d_next = noise_delta(normals4_pre(0u, ppre, &s_pt, s_rk), sigma);
                for (int j = 0; j < N; ++j) {
                    const unsigned g = g_run + (unsigned)j;
                    const int slot = slot_of(g);
                    const unsigned ph = (g / kRing) & 1u;
                    float4 d;
                    if (PIPE == 2) {
                        mbar_wait_or_abort(bar_of(slot, N_FULL), ph, abort_flag, wait_polls);
                        d = *nring_at(slot);
                        mbar_arrive(bar_of(slot, N_EMPTY));
                    } else {
                        d = d_next;
                        d_next = noise_delta(normals4_pre((unsigned)min(j + 1, N - 1), ppre, &s_pt, s_rk), sigma);
                    }
                    const float4 un = su[j];
                    const float4 u = clamp_input(Mdl, perturb(un, d));
                    const Feasible f = feasible(Mdl, x, u, inv_dt);
                    rk4(Mdl, x, cmp, f.Fm, f.tJx, f.tJy, f.tJz, dt);
                    // The tracking cost is formed here; the input and
                    // input-change cost by the cost lanes, from the control
                    // handed over with the position.
                    const float tcost = tracking_cost(C, x, cmp, &sref[4 * (j + 1)]);
                    if (g >= (unsigned)kRing) mbar_wait_or_abort(bar_of(slot, X_EMPTY), ph ^ 1u, abort_flag, wait_polls);
                    *ring_at(slot, 0) = make_float4(x.px, x.py, x.pz, tcost);
                    *ring_at(slot, 1) = make_float4(cmp.px, cmp.py, cmp.pz, 0.0f);
                    *ring_at(slot, 2) = u;
                    mbar_arrive(bar_of(slot, X_FULL));
                }
            } else {
                float S = 0.0f, Sc = 0.0f;
                int nhit = 0;
                bool hit = false;
                unsigned kept = 0;
                WarpList wl;
                wl.n = -1;
                kahan_add(S, Sc, tracking_cost(C, x, cmp, &sref[0]) +
                                     obstacle_cost<LANES>(C, x.px, x.py, x.pz, sobs, M, lane, wlane, wob, wl,
                                                          cull_margin, reuse_lists, &hit, &kept));
                if (C.grid) hit |= grid_hit(C, x.px + p0x, x.py + p0y, x.pz + p0z);
                nhit += hit ? 1 : 0;
                // Reads what was handed over for step j + 1 (slot sl):
                // returns the compensated position and the step's input,
                // input-change and tracking cost, in the one-thread form's
                // order.
                float4 u_prev = make_float4(0.f, 0.f, 0.f, 0.f);
                auto take = [&](int sl, int jj, float& qpx, float& qpy, float& qpz) -> float {
                    const float4 r0 = *ring_at(sl, 0), r1 = *ring_at(sl, 1);
                    float c;
                    if (PIPE == 3) {
                        c = r0.w;  // input, input-change and tracking cost, formed by the translation thread
                    } else {
                        const float4 u = *ring_at(sl, 2);
                        c = input_cost(C, u, u_prev, jj > 0);
                        u_prev = u;
                        c += r0.w;
                    }
                    qpx = r0.x - r1.x;
                    qpy = r0.y - r1.y;
                    qpz = r0.z - r1.z;
                    return c;
                };
                int j = 0;
                if (reuse_lists && M > 0) {
                    // kStatesPerPass states per pass over the kept list: the
                    // scoring is latency-bound, and several positions give
                    // each loaded obstacle that much more independent work.
                    // The sums are bitwise those of one state at a time
                    // (terms below the floor are 0 whichever box kept their
                    // obstacle).
                    constexpr int NS = kStatesPerPass;
                    for (; j + NS - 1 < N; j += NS) {
                        bool ok[NS];
                        float qx[NS], qy[NS], qz[NS], uc[NS];
                        bool all_ok = true;
#pragma unroll
                        for (int i = 0; i < NS; ++i) {
                            const unsigned g = g_run + (unsigned)(j + i);
                            const int sl = slot_of(g);
                            all_ok = all_ok && mbar_wait_or_abort(bar_of(sl, X_FULL), (g / kRing) & 1u, abort_flag,
                                                                  wait_polls);
                            ok[i] = all_ok;
                            uc[i] = take(sl, j + i, qx[i], qy[i], qz[i]);
                        }
#pragma unroll
                        for (int i = 0; i < NS; ++i) mbar_arrive(bar_of(slot_of(g_run + (unsigned)(j + i)), X_EMPTY));
                        float bars[NS];
                        bool hits[NS];
                        obstacle_cost_n<LANES, NS>(C, qx, qy, qz, sobs, M, lane, wlane, wob, wl, cull_margin, true,
                                                   bars, hits, &kept);
#pragma unroll
                        for (int i = 0; i < NS; ++i) {
                            bool h = hits[i];
                            if (C.grid) h |= grid_hit(C, qx[i] + p0x, qy[i] + p0y, qz[i] + p0z);
                            nhit += h ? 1 : 0;
                            kahan_add(S, Sc, (ok[i] ? uc[i] : NAN) + bars[i]);
                        }
                    }
                }
                for (; j < N; ++j) {
                    const unsigned g = g_run + (unsigned)j;
                    const int slot = slot_of(g);
                    const unsigned ph = (g / kRing) & 1u;
                    const bool ok = mbar_wait_or_abort(bar_of(slot, X_FULL), ph, abort_flag, wait_polls);
                    float qpx, qpy, qpz;  // compensated position
                    const float uc = take(slot, j, qpx, qpy, qpz);
                    mbar_arrive(bar_of(slot, X_EMPTY));
                    float step = ok ? uc : NAN;
                    step += obstacle_cost<LANES>(C, qpx, qpy, qpz, sobs, M, lane, wlane, wob, wl, cull_margin,
                                                 reuse_lists, &hit, &kept);
                    if (C.grid) hit |= grid_hit(C, qpx + p0x, qpy + p0y, qpz + p0z);
                    nhit += hit ? 1 : 0;
                    kahan_add(S, Sc, step);
                }
                if (a.stats) {
                    const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, valid && lane == 0));
                    if (wlane == 0 && kept) atomicAdd(a.stats, (unsigned long long)kept * nvalid);
                }
                if (lane == 0) {  // the cost lanes of a sample hold bitwise identical sums
                    const float2 Sk = cost_pair(C.c_obs, nhit, S, Sc);
                    if (valid && sI.costs) sI.costs[k_raw] = Sk.x;
                    sS[group] = (valid && isfinite(Sk.x)) ? Sk : make_float2(INFINITY, 0.0f);
                }
            }
            g_run += (unsigned)N;
            __syncthreads();
            if (s_abort && tid == 0) atomicOr(&a.errflags[inst], ERR_TIMEOUT);
        }

        // ------------------------------------- tile min, weights, eta_t
        // Sample g's cost is handled by thread g (spb <= nthreads), in the
        // first nsw warps.  rho_t: each of those warps reduces its 32 keys,
        // every thread takes the minimum of the warp minima.  Then each
        // sample's weight; per warp the contributors (weight > 0) by ballot
        // and the weight sum by a fixed shuffle tree; eta_t and the ascending
        // contributor list from the per-warp results in warp order.
        // With two samples per thread, sample r nthreads + tid belongs to
        // virtual warp r nwarps + warp (r = 0, 1): the virtual warps are the
        // samples' 32-aligned groups in ascending order.
        const int nsw = (spb + 31) >> 5;
#pragma unroll
        for (int r = 0; r < SPT; ++r) {
            const int vw = r * nwarps + warp, g = r * nthreads + tid;
            if (vw < nsw) {
                const unsigned long long kk = g < spb ? pair_key(sS[g]) : ~0ull;
                const unsigned long long m = warp_min_key(kk);
                if (wlane == 0) s_wkey[vw] = m;
            }
        }
        __syncthreads();
        unsigned long long mk = s_wkey[0];
        for (int w = 1; w < nsw; ++w) mk = min(mk, s_wkey[w]);
        const float2 rho_t = key_pair(mk);
        float e_own[SPT];
        unsigned rank[SPT];
#pragma unroll
        for (int r = 0; r < SPT; ++r) {
            const int vw = r * nwarps + warp, g = r * nthreads + tid;
            e_own[r] = 0.0f;
            rank[r] = 0;
            if (vw < nsw) {
                if (g < spb) {
                    e_own[r] = softmin_weight(sS[g], rho_t, lambda);
                    sE[g] = e_own[r];
                }
                const unsigned bal = __ballot_sync(0xffffffffu, e_own[r] > 0.0f);
                rank[r] = __popc(bal & ((1u << wlane) - 1u));
                const float ws = warp_sum(e_own[r]);
                if (wlane == 0) {
                    s_wcnt[vw] = __popc(bal);
                    s_red[vw] = ws;
                }
            }
        }
        __syncthreads();
        float eta_t = 0.0f;
        int count = 0, list_at[SPT];
#pragma unroll
        for (int r = 0; r < SPT; ++r) list_at[r] = 0;
        for (int w = 0; w < nsw; ++w) {
#pragma unroll
            for (int r = 0; r < SPT; ++r)
                if (w == r * nwarps + warp) list_at[r] = count;
            eta_t += s_red[w];
            count += s_wcnt[w];
        }
#pragma unroll
        for (int r = 0; r < SPT; ++r)
            if (e_own[r] > 0.0f) slist[list_at[r] + (int)rank[r]] = r * nthreads + tid;
        __syncthreads();

        // ---------------------- weighted sum of the regenerated noise
        // Threads (j, grp): grp-th share of the contributors for step j.
        {
            const int G = N >= nthreads ? 1 : nthreads / N;
            const int tile_base = tile * spb;
            for (int w = tid; w < (N >= nthreads ? N : G * N); w += nthreads) {
                const int j = w % N, grp = w / N;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int ci = grp; ci < count; ci += G) {
                    const int g = slist[ci];
                    const float e = sE[g];
                    const float4 d = noise_delta(normals4((unsigned)(tile_base + g), (unsigned)j, iter, s_rk), sigma);
                    acc.x = fmaf(e, d.x, acc.x);
                    acc.y = fmaf(e, d.y, acc.y);
                    acc.z = fmaf(e, d.z, acc.z);
                    acc.w = fmaf(e, d.w, acc.w);
                }
                spart[grp * N + j] = acc;
            }
            __syncthreads();
            float* P = a.partials + sI.part_off + (long long)tile * partial_stride(N);
            for (int j = tid; j < N; j += nthreads) {
                float4 s = spart[j];
                for (int grp = 1; grp < G; ++grp) {
                    const float4 t = spart[grp * N + j];
                    s.x += t.x; s.y += t.y; s.z += t.z; s.w += t.w;
                }
                reinterpret_cast<float4*>(P + 4)[j] = s;
            }
            if (tid == 0) {
                P[0] = rho_t.x;
                P[1] = rho_t.y;
                P[2] = eta_t;
                P[3] = 0.0f;
            }
        }

        // ----------------------------- last tile of the instance merges
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&a.done[inst], 1u);
            s_last = (prev == (unsigned)(sI.n_tiles - 1)) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const int T = sI.n_tiles;
            const int stride = partial_stride(N);
            const float* P0 = a.partials + sI.part_off;
            // When the instance has at most spb tiles, every tile's header
            // (rho_t, eta_t) is read once into shared memory and the merge
            // scales s_t stay there; otherwise they go through the partials.
            const bool fast = T <= spb;
            // rho = min rho_t (the cost-pair header of each partial): per
            // thread, per warp by key, then every thread over the warps.
            unsigned long long mk = ~0ull;
            for (int t = tid; t < T; t += nthreads) {
                const float2 rt = __ldcg(reinterpret_cast<const float2*>(P0 + (long long)t * stride));
                if (fast) {
                    sS[t] = rt;
                    sE[t] = __ldcg(P0 + (long long)t * stride + 2);
                }
                mk = min(mk, pair_key(rt));
            }
            mk = warp_min_key(mk);
            if (wlane == 0) s_wkey[warp] = mk;
            __syncthreads();
            mk = s_wkey[0];
            for (int w = 1; w < nwarps; ++w) mk = min(mk, s_wkey[w]);
            const float2 rho = key_pair(mk);
            // s_t = exp(-(rho_t - rho)/lambda), kept in shared memory (fast)
            // or in the partial's pad slot; eta = sum_t s_t eta_t (per warp
            // by a shuffle tree, then over the warps in order).
            float* Pw = a.partials + sI.part_off;
            float eacc = 0.0f;
            for (int t = tid; t < T; t += nthreads) {
                const float2 rt = fast ? sS[t] : __ldcg(reinterpret_cast<const float2*>(P0 + (long long)t * stride));
                const float et = fast ? sE[t] : __ldcg(P0 + (long long)t * stride + 2);
                const float st = softmin_weight(rt, rho, lambda);
                if (fast) sE[t] = st;
                else __stcg(Pw + (long long)t * stride + 3, st);
                eacc = fmaf(st, et, eacc);
            }
            eacc = warp_sum(eacc);
            if (wlane == 0) s_red[warp] = eacc;
            __syncthreads();
            float eta = 0.0f;
            for (int w = 0; w < nwarps; ++w) eta += s_red[w];
            const bool ok = rho.x < INFINITY && eta > 0.0f;
            const unsigned errs = a.errflags[inst];
            // u_out = u_nom + Sigma / eta   (Eq. u_update), Sigma = sum_t
            // s_t Sigma_t.  The tiles with s_t > 0 are compacted, in
            // ascending order and a chunk of spb tiles at a time, into shared
            // memory; threads (j, grp) add the grp-th share of them for step
            // j (independent loads, so they overlap), and the shares are then
            // added in group order.
            float* sunew = reinterpret_cast<float*>(su);
            const int G = N >= nthreads ? 1 : nthreads / N;
            for (int w0 = 0; ok && w0 < G * N; w0 += nthreads) {
                const int w = w0 + tid;
                const int j = w % N, grp = w / N;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int t0 = 0; t0 < T; t0 += spb) {
                    const int ch = min(spb, T - t0);
                    if (!fast)
                        for (int i = tid; i < ch; i += nthreads) sE[i] = __ldcg(P0 + (long long)(t0 + i) * stride + 3);
                    __syncthreads();
                    if (warp == 0) {
                        int base = 0;
                        for (int c0 = 0; c0 < ch; c0 += 32) {
                            const int i = c0 + wlane;
                            const bool on = i < ch && sE[i] > 0.0f;
                            const unsigned bal = __ballot_sync(0xffffffffu, on);
                            if (on) slist[base + __popc(bal & ((1u << wlane) - 1u))] = i;
                            base += __popc(bal);
                        }
                        if (wlane == 0) s_count = base;
                    }
                    __syncthreads();
                    const int cnt = s_count;
                    if (w < G * N) {
#pragma unroll 4
                        for (int ci = grp; ci < cnt; ci += G) {
                            const int i = slist[ci];
                            const float st = sE[i];
                            const float4 v =
                                __ldcg(reinterpret_cast<const float4*>(P0 + (long long)(t0 + i) * stride + 4) + j);
                            acc.x = fmaf(st, v.x, acc.x);
                            acc.y = fmaf(st, v.y, acc.y);
                            acc.z = fmaf(st, v.z, acc.z);
                            acc.w = fmaf(st, v.w, acc.w);
                        }
                    }
                    __syncthreads();
                }
                if (w < G * N) spart[grp * N + j] = acc;
            }
            __syncthreads();
            for (int j = tid; j < N; j += nthreads) {
                float4 sg = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ok) {
                    sg = spart[j];
                    for (int grp = 1; grp < G; ++grp) {
                        const float4 t = spart[grp * N + j];
                        sg.x += t.x; sg.y += t.y; sg.z += t.z; sg.w += t.w;
                    }
                }
                const float acc[4] = {sg.x, sg.y, sg.z, sg.w};
                // u_nom_j as staged in shared memory (sunew aliases it; this
                // thread reads its row before it overwrites it).
                const float4 un4 = su[j];
                const float unj[4] = {un4.x, un4.y, un4.z, un4.w};
                for (int c = 0; c < 4; ++c) {
                    const int o = 4 * j + c;
                    const float un = unj[c];
                    const float v = ok ? un + acc[c] / eta : un;
                    sunew[o] = v;
                    if (sI.u_out) sI.u_out[o] = v;
                }
            }
            // ApplyToSystem(u_nom_0) by the thread that formed u_out_0
            // (j = 0 above), while the others go on to the warm start.
            if (tid == 0) {
                // ApplyToSystem(u_nom_0): feasible command from x_hat.
                State xh;
                xh.px = s_xhat[0]; xh.py = s_xhat[1]; xh.pz = s_xhat[2]; xh.qw = s_xhat[3];
                xh.qx = s_xhat[4]; xh.qy = s_xhat[5]; xh.qz = s_xhat[6]; xh.vx = s_xhat[7];
                xh.vy = s_xhat[8]; xh.vz = s_xhat[9]; xh.wx = s_xhat[10]; xh.wy = s_xhat[11];
                xh.wz = s_xhat[12];
                const float4 u0 = clamp_input(Mdl, make_float4(sunew[0], sunew[1], sunew[2], sunew[3]));
                const Feasible f = feasible(Mdl, xh, u0, inv_dt);
                if (sI.u_cmd) {
                    sI.u_cmd[0] = f.F;
                    sI.u_cmd[1] = xh.wx + (f.tx - f.gx) * Mdl.inv_Jx * dt;
                    sI.u_cmd[2] = xh.wy + (f.ty - f.gy) * Mdl.inv_Jy * dt;
                    sI.u_cmd[3] = xh.wz + (f.tz - f.gz) * Mdl.inv_Jz * dt;
                }
                if (sI.x_next) {
                    rk4(Mdl, xh, f.Fm, f.tJx, f.tJy, f.tJz,
                        C.shift_alpha * dt);
                    const float v[13] = {xh.px, xh.py, xh.pz, xh.qw, xh.qx, xh.qy, xh.qz,
                                         xh.vx, xh.vy, xh.vz, xh.wx, xh.wy, xh.wz};
                    for (int i = 0; i < 13; ++i) sI.x_next[i] = v[i];
                }
                int st = MPPI_OK;
                if (errs & ERR_TIMEOUT) st = MPPI_ETIMEOUT;
                else if (!ok) st = MPPI_ENONFINITE;
                if (sI.status) *sI.status = st;
                if (sI.iter_dev) *sI.iter_dev = iter + 1ull;
                a.done[inst] = 0u;
                a.errflags[inst] = 0u;
            }
            __syncthreads();
            // Warm start: shift by alpha steps with linear interpolation.
            if (sI.u_next) {
                const float al = C.shift_alpha;
                for (int o = tid; o < 4 * N; o += nthreads) {
                    const int j = o >> 2, c = o & 3;
                    const float later = (j + 1 < N) ? sunew[o + 4] : (C.tail_mode == 1 ? sunew[o] : Mdl.u_init[c]);
                    sI.u_next[o] = al == 1.0f ? later : fmaf(al, later - sunew[o], sunew[o]);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- host

// One thread per sample in blocks of at most 128 threads (the batched
// launches' default) runs the instantiation that fits 6 blocks per SM: 24
// warps instead of 16 raise the issue rate of these issue-bound launches
// (256 uneven instances: 7.52 -> 7.23 ms; at most 85 registers, no spills).
constexpr int kMinBlocks128 = 6;
// Two samples per thread (blocks of 64 or 128 threads): compiled for 4
// blocks of 128 per SM, a budget of 128 registers a thread.
constexpr int kMinBlocksX2 = 4;

bool shape_supported(Shape s) {
    if (s.spt == 2) return s.pipe == 0 && s.lanes == 1 && (s.block == 64 || s.block == 128);
    if (s.spt != 1) return false;
    if (s.pipe >= 1 && s.pipe <= 3) {
        // A dynamics warp (pipe 2: and a noise warp; pipe 3: an attitude, a
        // noise and a translation warp) plus `lanes` cost warps per 32
        // samples.
        const int unit = 32 * (s.pipe + s.lanes);
        return (s.lanes == 1 || s.lanes == 2) && s.block >= unit && s.block <= 512 && s.block % unit == 0;
    }
    const bool lanes_ok = s.lanes == 1 || s.lanes == 2 || s.lanes == 4 || s.lanes == 8 || s.lanes == 32;
    const bool block_ok = s.block == 64 || s.block == 128 || s.block == 256 || s.block == 512;
    return s.pipe == 0 && lanes_ok && block_ok;
}

size_t smem_bytes(int N_max, int M_max, Shape s) {
    return smem_layout(N_max, M_max, s.block, s.lanes, s.pipe, s.spt).total;
}

// Largest dynamic shared memory opted in so far, per instantiation and per
// device (the attribute belongs to the device's context).  The attribute is
// raised only when a launch needs more, so launches that are being captured
// into a graph (after a first, uncaptured preparation) make no attribute
// call.
constexpr int kMaxDevices = 64;

template <int LANES, int PIPE, int MINB, int SPT>
static std::atomic<int>* smem_opt_in() {
    static std::atomic<int> v[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;  // unknown device: set the attribute every time
    }
    return &v[dev];
}

template <int LANES, int PIPE, int MINB, int SPT>
static cudaError_t prepare_t(size_t smem) {
    std::atomic<int>* opt = smem_opt_in<LANES, PIPE, MINB, SPT>();
    if (opt && (int)smem <= opt->load()) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mppi_step_kernel<LANES, PIPE, MINB, SPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && opt) {
        int cur = opt->load();
        while ((int)smem > cur && !opt->compare_exchange_weak(cur, (int)smem)) {
        }
    }
    return e;
}

template <int LANES, int PIPE, int MINB = 1, int SPT = 1>
static cudaError_t launch_t(const LaunchArgs& a, int block, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = prepare_t<LANES, PIPE, MINB, SPT>(smem);
    if (e != cudaSuccess) return e;
    mppi_step_kernel<LANES, PIPE, MINB, SPT><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tiles(const LaunchArgs& args, Shape s, int grid, size_t smem, cudaStream_t st) {
    LaunchArgs a = args;
    a.C.cull_margin = list_margin(s);
    if (s.spt == 2) return launch_t<1, 0, kMinBlocksX2, 2>(a, s.block, grid, smem, st);
    if (s.pipe == 1) {
        if (s.lanes == 1) return launch_t<1, 1>(a, s.block, grid, smem, st);
        if (s.lanes == 2) return launch_t<2, 1>(a, s.block, grid, smem, st);
        return cudaErrorInvalidValue;
    }
    if (s.pipe == 2) {
        if (s.lanes == 1) return launch_t<1, 2>(a, s.block, grid, smem, st);
        if (s.lanes == 2) return launch_t<2, 2>(a, s.block, grid, smem, st);
        return cudaErrorInvalidValue;
    }
    if (s.pipe == 3) {
        if (s.lanes == 1) return launch_t<1, 3>(a, s.block, grid, smem, st);
        if (s.lanes == 2) return launch_t<2, 3>(a, s.block, grid, smem, st);
        return cudaErrorInvalidValue;
    }
    switch (s.lanes) {
        case 1:
            return s.block <= 128 ? launch_t<1, 0, kMinBlocks128>(a, s.block, grid, smem, st)
                                  : launch_t<1, 0>(a, s.block, grid, smem, st);
        case 2: return launch_t<2, 0>(a, s.block, grid, smem, st);
        case 4: return launch_t<4, 0>(a, s.block, grid, smem, st);
        case 8: return launch_t<8, 0>(a, s.block, grid, smem, st);
        case 32: return launch_t<32, 0>(a, s.block, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int LANES, int PIPE, int MINB = 1, int SPT = 1>
static int occupancy_t(int block, size_t smem) {
    int n = 0;
    prepare_t<LANES, PIPE, MINB, SPT>(smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mppi_step_kernel<LANES, PIPE, MINB, SPT>, block, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

int max_active_blocks(Shape s, size_t smem) {
    if (s.spt == 2) return occupancy_t<1, 0, kMinBlocksX2, 2>(s.block, smem);
    if (s.pipe == 1) return s.lanes == 2 ? occupancy_t<2, 1>(s.block, smem) : occupancy_t<1, 1>(s.block, smem);
    if (s.pipe == 2) return s.lanes == 2 ? occupancy_t<2, 2>(s.block, smem) : occupancy_t<1, 2>(s.block, smem);
    if (s.pipe == 3) return s.lanes == 2 ? occupancy_t<2, 3>(s.block, smem) : occupancy_t<1, 3>(s.block, smem);
    switch (s.lanes) {
        case 1:
            return s.block <= 128 ? occupancy_t<1, 0, kMinBlocks128>(s.block, smem)
                                  : occupancy_t<1, 0>(s.block, smem);
        case 2: return occupancy_t<2, 0>(s.block, smem);
        case 4: return occupancy_t<4, 0>(s.block, smem);
        case 8: return occupancy_t<8, 0>(s.block, smem);
        case 32: return occupancy_t<32, 0>(s.block, smem);
        default: return 1;
    }
}

// The sampling step alone: delta for samples k0 .. k0 + K - 1, steps
// 0 .. N - 1, element e = (k - k0) N + j, by the device functions the
// rollouts call (same counters, keys and rounding, so the same bits).
__global__ void __launch_bounds__(256) noise_kernel(float4* out, unsigned k0, int K, int N,
                                                    unsigned long long iter, unsigned key0, unsigned key1,
                                                    float4 sig) {
    uint4 rk[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) rk[i] = philox_round_keys(key0, key1, (unsigned)i);
    const uint2 pt = philox_pre_tile(iter, rk);
    const float sigma[4] = {sig.x, sig.y, sig.z, sig.w};
    const long long total = (long long)K * N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const long long kk = e / N;
        const unsigned j = (unsigned)(e - kk * N);
        const PhiloxPre pp = philox_pre_sample(k0 + (unsigned)kk, iter, rk);
        out[e] = noise_delta(normals4_pre(j, pp, &pt, rk), sigma);
    }
}

cudaError_t launch_noise(float* out, unsigned k0, int K, int N, unsigned long long iter, unsigned key0,
                         unsigned key1, const float* sigma, cudaStream_t st) {
    const long long total = (long long)K * N;
    const long long blocks = (total + 255) / 256;
    const long long cap = 8ll * sm_count();
    const int grid = (int)(blocks < cap ? blocks : cap);
    noise_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<float4*>(out), k0, K, N, iter, key0, key1,
                                       make_float4(sigma[0], sigma[1], sigma[2], sigma[3]));
    return cudaGetLastError();
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace mppi
