/*
 * mppi_oracle.c -- plain, slow, FP64 CPU implementation of one MPPI
 * optimisation step for the quadrotor of "Model Predictive Path Integral
 * Control for Agile Unmanned Aerial Vehicles" (Minarik, Penicka, Vonasek,
 * Saska; arXiv 2407.09812).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle against which the CUDA
 * path is checked.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA path; the only thing both sides share is
 * the seeded input generator (which holds none of the method's arithmetic).
 *
 * Every function follows one passage of the paper, cited in its comment,
 * in the paper's order and notation.  Where the paper is silent the reading
 * taken is stated beside the code ("Reading:").  No blocking, fusion or
 * reordering is done beyond what the equations state: each equation is one
 * plain loop so that it can be checked against the paper by eye.
 *
 * Conventions (readings where the paper is silent):
 *   state x = [p(3), q(4) = (w, x, y, z), v(3), omega(3)], world z up,
 *   gravity g = (0, 0, -g); q rotates body to world; Hamilton product.
 *   control u = [F_t, omega_xd, omega_yd, omega_zd].
 *   obstacle = (cx, cy, cz, r); r >= 0 sphere, r < 0 vertical infinite
 *   cylinder of radius |r| (cz unused).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENONFINITE (-5)

typedef struct {
    double mass;       /* m  [kg], Table I                                  */
    double g;          /* |g| [m/s^2]                                        */
    double arm_l;      /* l  [m], Table I                                    */
    double c_tf;       /* rotor torque constant [m], Table I                 */
    double J[3];       /* diagonal inertia [kg m^2], Table I                 */
    double T_min;      /* per-rotor thrust limits [N], Table I               */
    double T_max;
    int motor_clip;    /* 1: clip rotor thrusts (Eq. clipping)               */
    int pad0;
    double F_min;      /* safety box on the desired collective thrust [N]    */
    double F_max;
    double w_max[3];   /* safety box on desired body rates [rad/s] (Sec. IV) */
} orc_model;

typedef struct {
    int K, N;          /* rollouts, prediction steps                         */
    double dt;         /* prediction time step [s]                           */
    double lambda;     /* temperature of Eq. cost_2                          */
    double sigma[4];   /* standard deviation of each control component      */
    double c_p, c_q, c_v, c_w;   /* Eq. rho_ref weights                      */
    double R[4], Rd[4];          /* Eq. cost diagonal weights                */
    double c_obs;      /* collision indicator weight (Sec. IV-D)             */
    double c_bar;      /* exponential barrier weight (reading)               */
    double beta;       /* barrier rate [1/m^2] (reading)                     */
    double r_uav;      /* vehicle radius added to each obstacle [m]          */
    int quat_metric;   /* 0: Eq. quat_approx, 1: Eq. quat_angle              */
    int tail_mode;     /* 0: last control re-initialised, 1: repeated        */
    double shift_alpha;/* 1: shift by one step (Alg. 1); (0,1): Sec. IV-B    */
    double delay;      /* >0: delay compensation by prediction (Sec. IV-E)   */
    uint64_t seed;
    uint32_t stream_id;
    int pad1;
    /* Occupancy voxel grid (a grid-based collision module, Sec. IV-D):
     * grid[(iz * gy + iy) * gx + ix] != 0 marks an occupied voxel of edge
     * g_voxel whose lowest corner is g_origin + voxel * (ix, iy, iz);
     * positions outside the grid are free.  grid == NULL: no grid. */
    const uint8_t* grid;
    int gx, gy, gz, pad2;
    double g_origin[3];
    double g_voxel;
} orc_params;

/* ------------------------------------------------------------------------
 * Noise: delta u_j^k ~ N(0, Sigma) (Sec. III-A, Eq. rollout_computation).
 *
 * Counter-based generator Philox4x32-10 from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2,
 * 3", SC 2011): ten rounds; in each round words 0 and 2 are multiplied by
 * the two round multipliers giving 64-bit products; the new words are
 * (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); after
 * every round the key words are bumped by the two Weyl constants.
 * Reading: counter = (k, j, iter_lo, iter_hi), key = (seed_lo,
 * seed_hi ^ stream_id).
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0,1) from the top 23 bits of a word:
 * (2 m + 1) 2^-24 with m = r >> 9.  Exactly representable in FP32 and FP64. */
double orc_uniform(uint32_t r)
{
    return (2.0 * (double)(r >> 9) + 1.0) * (1.0 / 16777216.0);
}

/* Box & Muller (1958): two independent standard normals from two uniforms. */
void orc_box_muller(double u0, double u1, double* z0, double* z1)
{
    const double two_pi = 6.283185307179586476925286766559;
    double radius = sqrt(-2.0 * log(u0));
    *z0 = radius * cos(two_pi * u1);
    *z1 = radius * sin(two_pi * u1);
}

/* delta u_j^k = sigma o z, z ~ N(0, I) (Sigma diagonal, reading). */
void orc_noise(const orc_params* P, uint64_t iter, uint32_t k, uint32_t j, double delta[4])
{
    uint32_t ctr[4] = {k, j, (uint32_t)(iter & 0xffffffffu), (uint32_t)(iter >> 32)};
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu),
                       (uint32_t)(P->seed >> 32) ^ P->stream_id};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double z[4];
    orc_box_muller(orc_uniform(r[0]), orc_uniform(r[1]), &z[0], &z[1]);
    orc_box_muller(orc_uniform(r[2]), orc_uniform(r[3]), &z[2], &z[3]);
    for (int c = 0; c < 4; ++c) delta[c] = P->sigma[c] * z[c];
}

/* ------------------------------------------------------------------------
 * Model (Sec. III-B, Eq. drone_dynamics).
 * ---------------------------------------------------------------------- */

/* Hamilton product a (.) b, quaternions as (w, x, y, z). */
void orc_quat_mul(const double a[4], const double b[4], double out[4])
{
    out[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    out[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    out[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    out[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* R(q): rotation matrix of a unit quaternion (body to world), row major. */
void orc_rotation_matrix(const double q[4], double Rm[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    Rm[0] = 1.0 - 2.0 * (y * y + z * z);
    Rm[1] = 2.0 * (x * y - w * z);
    Rm[2] = 2.0 * (x * z + w * y);
    Rm[3] = 2.0 * (x * y + w * z);
    Rm[4] = 1.0 - 2.0 * (x * x + z * z);
    Rm[5] = 2.0 * (y * z - w * x);
    Rm[6] = 2.0 * (x * z - w * y);
    Rm[7] = 2.0 * (y * z + w * x);
    Rm[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* x_dot = f(x, F_t, tau), Eq. drone_dynamics:
 *   p_dot = v,  q_dot = 1/2 q (.) [0, omega],
 *   v_dot = 1/m R(q) [0, 0, F_t] + g,  omega_dot = J^-1 (tau - omega x J omega). */
void orc_dynamics(const orc_model* Mdl, const double x[13], double F_t, const double tau[3],
                  double xdot[13])
{
    const double* q = &x[3];
    const double* v = &x[7];
    const double* w = &x[10];

    for (int i = 0; i < 3; ++i) xdot[i] = v[i];

    double w_quat[4] = {0.0, w[0], w[1], w[2]};
    double qw[4];
    orc_quat_mul(q, w_quat, qw);
    for (int i = 0; i < 4; ++i) xdot[3 + i] = 0.5 * qw[i];

    double Rm[9];
    orc_rotation_matrix(q, Rm);
    double thrust_body[3] = {0.0, 0.0, F_t};
    double gravity[3] = {0.0, 0.0, -Mdl->g};
    for (int r = 0; r < 3; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 3; ++c) acc += Rm[3 * r + c] * thrust_body[c];
        xdot[7 + r] = acc / Mdl->mass + gravity[r];
    }

    double Jw[3] = {Mdl->J[0] * w[0], Mdl->J[1] * w[1], Mdl->J[2] * w[2]};
    double wxJw[3];
    cross3(w, Jw, wxJw);
    for (int i = 0; i < 3; ++i) xdot[10 + i] = (tau[i] - wxJw[i]) / Mdl->J[i];
}

/* x_{j+1} = x_j + f_RK4(x_j, u_j, dt) (Eq. rollout_computation): the
 * classical four-stage Runge-Kutta step, inputs (F_t, tau) held over the
 * step (reading: zero-order hold).  Reading: the quaternion is
 * renormalised after the step so that ||q|| = 1 holds (Sec. III-B). */
void orc_rk4_step(const orc_model* Mdl, const double x[13], double F_t, const double tau[3],
                  double h, double x_next[13])
{
    double k1[13], k2[13], k3[13], k4[13], xs[13];
    orc_dynamics(Mdl, x, F_t, tau, k1);
    for (int i = 0; i < 13; ++i) xs[i] = x[i] + 0.5 * h * k1[i];
    orc_dynamics(Mdl, xs, F_t, tau, k2);
    for (int i = 0; i < 13; ++i) xs[i] = x[i] + 0.5 * h * k2[i];
    orc_dynamics(Mdl, xs, F_t, tau, k3);
    for (int i = 0; i < 13; ++i) xs[i] = x[i] + h * k3[i];
    orc_dynamics(Mdl, xs, F_t, tau, k4);
    for (int i = 0; i < 13; ++i)
        x_next[i] = x[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    double n = sqrt(x_next[3] * x_next[3] + x_next[4] * x_next[4] + x_next[5] * x_next[5] +
                    x_next[6] * x_next[6]);
    for (int i = 3; i < 7; ++i) x_next[i] /= n;
}

/* ------------------------------------------------------------------------
 * Low-level constraints (Sec. III-B, equations after Eq. drone_dynamics).
 * ---------------------------------------------------------------------- */

/* Allocation matrix Gamma (Sec. III-B), row major, rows (F_t, tau_x,
 * tau_y, tau_z), columns rotors 1..4. */
void orc_allocation_matrix(const orc_model* Mdl, double G[16])
{
    double a = Mdl->arm_l / sqrt(2.0);
    double c = Mdl->c_tf;
    double rows[16] = {1.0, 1.0, 1.0, 1.0,
                       -a,  a,   a,   -a,
                       -a,  a,   -a,  a,
                       -c,  -c,  c,   c};
    memcpy(G, rows, sizeof(rows));
}

/* Inverse of a 4x4 matrix by Gauss-Jordan elimination with partial
 * pivoting (textbook).  Returns 0 on success, -1 if singular. */
int orc_invert4(const double A[16], double Ainv[16])
{
    double m[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c) m[r][c] = c < 4 ? A[4 * r + c] : (c - 4 == r ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
        if (m[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 8; ++c) { double t = m[col][c]; m[col][c] = m[piv][c]; m[piv][c] = t; }
        double d = m[col][col];
        for (int c = 0; c < 8; ++c) m[col][c] /= d;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            double f = m[r][col];
            for (int c = 0; c < 8; ++c) m[r][c] -= f * m[col][c];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) Ainv[4 * r + c] = m[r][c + 4];
    return 0;
}

/* Safety limits on the desired control (Sec. IV, omega_xy,max and
 * omega_z,max; collective-thrust range): u clamped into the box. */
void orc_clamp_input(const orc_model* Mdl, const double u_in[4], double u_out[4])
{
    double F = u_in[0];
    if (F < Mdl->F_min) F = Mdl->F_min;
    if (F > Mdl->F_max) F = Mdl->F_max;
    u_out[0] = F;
    for (int i = 0; i < 3; ++i) {
        double w = u_in[1 + i];
        if (w < -Mdl->w_max[i]) w = -Mdl->w_max[i];
        if (w > Mdl->w_max[i]) w = Mdl->w_max[i];
        u_out[1 + i] = w;
    }
}

/* Feasible input from the desired u_d = [F_t, omega_d] at state x over
 * the time step dt (Sec. III-B):
 *   omega_dot_d = (omega_d - omega) / dt
 *   tau_d       = J omega_dot_d + omega x J omega
 *   T_d         = Gamma^-1 [F_t; tau_d]
 *   T_clip      = clip(T_min, T_d, T_max)                (Eq. clipping)
 *   [F_clip; tau_clip] = Gamma T_clip                   (Eq. clipped_torque_colthrust)
 *   omega_dot_clip = J^-1 (tau_clip - omega x J omega)
 *   omega_clip     = omega + omega_dot_clip dt          (Eq. clipped_states)
 * With motor_clip == 0 the clip step is the identity. */
void orc_feasible_input(const orc_model* Mdl, const double x[13], const double u_d[4], double dt,
                        double* F_clip, double tau_clip[3], double w_clip[3])
{
    const double* w = &x[10];
    double w_dot_d[3];
    for (int i = 0; i < 3; ++i) w_dot_d[i] = (u_d[1 + i] - w[i]) / dt;

    double Jw[3] = {Mdl->J[0] * w[0], Mdl->J[1] * w[1], Mdl->J[2] * w[2]};
    double wxJw[3];
    cross3(w, Jw, wxJw);
    double tau_d[3];
    for (int i = 0; i < 3; ++i) tau_d[i] = Mdl->J[i] * w_dot_d[i] + wxJw[i];

    double G[16], Ginv[16];
    orc_allocation_matrix(Mdl, G);
    orc_invert4(G, Ginv);
    double wrench_d[4] = {u_d[0], tau_d[0], tau_d[1], tau_d[2]};
    double T_d[4];
    for (int r = 0; r < 4; ++r) {
        T_d[r] = 0.0;
        for (int c = 0; c < 4; ++c) T_d[r] += Ginv[4 * r + c] * wrench_d[c];
    }

    double T_clip[4];
    for (int r = 0; r < 4; ++r) {
        double T = T_d[r];
        if (Mdl->motor_clip) {
            if (T < Mdl->T_min) T = Mdl->T_min;
            if (T > Mdl->T_max) T = Mdl->T_max;
        }
        T_clip[r] = T;
    }

    double wrench_clip[4];
    for (int r = 0; r < 4; ++r) {
        wrench_clip[r] = 0.0;
        for (int c = 0; c < 4; ++c) wrench_clip[r] += G[4 * r + c] * T_clip[c];
    }
    *F_clip = wrench_clip[0];
    for (int i = 0; i < 3; ++i) tau_clip[i] = wrench_clip[1 + i];

    for (int i = 0; i < 3; ++i) {
        double w_dot_clip = (tau_clip[i] - wxJw[i]) / Mdl->J[i];
        w_clip[i] = w[i] + w_dot_clip * dt;
    }
}

/* ------------------------------------------------------------------------
 * Cost (Sec. IV-C, Eq. cost, Eq. rho_ref, Eq. quat_approx / quat_angle;
 * Sec. IV-D obstacle term).
 * ---------------------------------------------------------------------- */

/* d_q(q1, q2): metric 0 -> 1 - <q1,q2>^2 (Eq. quat_approx);
 *              metric 1 -> acos(2 <q1,q2>^2 - 1) (Eq. quat_angle). */
double orc_quat_distance(const double q1[4], const double q2[4], int metric)
{
    double dot = q1[0] * q2[0] + q1[1] * q2[1] + q1[2] * q2[2] + q1[3] * q2[3];
    if (metric == 0) return 1.0 - dot * dot;
    double c = 2.0 * dot * dot - 1.0;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return acos(c);
}

/* rho_ref(x, x_ref) = c_p ||p - p_ref||^2 + c_q d_q(q, q_ref)^2
 *                   + c_v ||v - v_ref||^2 + c_w ||omega - omega_ref||^2. */
double orc_rho_ref(const orc_params* P, const double x[13], const double ref[13])
{
    double dp = 0.0, dv = 0.0, dw = 0.0;
    for (int i = 0; i < 3; ++i) {
        dp += (x[i] - ref[i]) * (x[i] - ref[i]);
        dv += (x[7 + i] - ref[7 + i]) * (x[7 + i] - ref[7 + i]);
        dw += (x[10 + i] - ref[10 + i]) * (x[10 + i] - ref[10 + i]);
    }
    double dq = orc_quat_distance(&x[3], &ref[3], P->quat_metric);
    return P->c_p * dp + P->c_q * dq * dq + P->c_v * dv + P->c_w * dw;
}

/* ||u||_R^2 with R diagonal (Eq. cost). */
double orc_input_cost(const orc_params* P, const double u[4])
{
    double s = 0.0;
    for (int c = 0; c < 4; ++c) s += P->R[c] * u[c] * u[c];
    return s;
}

/* ||u_{j+1} - u_j||_{R_Delta}^2 with R_Delta diagonal (Eq. cost). */
double orc_rate_cost(const orc_params* P, const double u_prev[4], const double u[4])
{
    double s = 0.0;
    for (int c = 0; c < 4; ++c) s += P->Rd[c] * (u[c] - u_prev[c]) * (u[c] - u_prev[c]);
    return s;
}

/* Signed squared gap of the position p to obstacle o (reading): sphere
 * ||p - c||^2 - (r + r_uav)^2; vertical cylinder (r < 0) the same in the
 * horizontal plane with radius |r|.  Negative or zero means collision. */
double orc_obstacle_gap(const orc_params* P, const double p[3], const double o[4])
{
    double r = o[3] < 0.0 ? -o[3] : o[3];
    double reach = r + P->r_uav;
    double dx = p[0] - o[0], dy = p[1] - o[1], dz = p[2] - o[2];
    double d2 = o[3] < 0.0 ? dx * dx + dy * dy : dx * dx + dy * dy + dz * dz;
    return d2 - reach * reach;
}

/* Voxel of position p in the occupancy grid: 1 if occupied, 0 if free or
 * outside.  *face_gap (optional) gets the distance from p to the nearest
 * face of its voxel across which occupancy changes (+inf if none), used
 * by tests to flag positions on an occupancy boundary. */
int orc_grid_occupied(const orc_params* P, const double p[3], double* face_gap)
{
    if (!P->grid) return 0;
    int n[3] = {P->gx, P->gy, P->gz};
    int idx[3];
    double frac[3];
    for (int a = 0; a < 3; ++a) {
        double c = (p[a] - P->g_origin[a]) / P->g_voxel;
        double f = floor(c);
        idx[a] = (int)f;
        frac[a] = c - f;
    }
    int inside = 1;
    for (int a = 0; a < 3; ++a)
        if (idx[a] < 0 || idx[a] >= n[a]) inside = 0;
    int occ = inside ? P->grid[((size_t)idx[2] * P->gy + idx[1]) * P->gx + idx[0]] != 0 : 0;
    if (face_gap) {
        double best = INFINITY;
        for (int a = 0; a < 3; ++a) {
            for (int side = 0; side < 2; ++side) {
                int nb[3] = {idx[0], idx[1], idx[2]};
                nb[a] += side ? 1 : -1;
                int nb_in = nb[0] >= 0 && nb[0] < n[0] && nb[1] >= 0 && nb[1] < n[1] && nb[2] >= 0 && nb[2] < n[2];
                int nb_occ = nb_in ? P->grid[((size_t)nb[2] * P->gy + nb[1]) * P->gx + nb[0]] != 0 : 0;
                if (nb_occ != occ) {
                    double d = (side ? 1.0 - frac[a] : frac[a]) * P->g_voxel;
                    if (d < best) best = d;
                }
            }
        }
        *face_gap = best;
    }
    return occ;
}

/* Obstacle cost of one state (Sec. IV-D): c_obs * 1[x in C_obs] (one
 * indicator per state), plus the exponential barrier of the reading
 * c_bar * exp(-beta * max(gap, 0)) summed over obstacles.
 * *min_gap (test instrumentation, not part of the cost) gets the smaller of
 * itself and this state's distance from the indicator's discontinuity: the
 * indicator flips where the state's smallest gap over the obstacles
 * crosses 0, so that distance is |smallest gap| (and, with a grid, the
 * distance to the nearest voxel face across which occupancy changes).
 * Tests use it to flag samples with a state on a collision boundary. */
double orc_obstacle_cost(const orc_params* P, const double x[13], const double* obs, int M,
                         double* min_gap)
{
    double barrier = 0.0;
    int in_collision = 0;
    double smallest = INFINITY;
    for (int o = 0; o < M; ++o) {
        double s = orc_obstacle_gap(P, x, &obs[4 * o]);
        if (s < smallest) smallest = s;
        barrier += P->c_bar * exp(-P->beta * (s > 0.0 ? s : 0.0));
        if (s <= 0.0) in_collision = 1;
    }
    double edge = fabs(smallest);
    if (P->grid) {
        double face = INFINITY;
        if (orc_grid_occupied(P, x, &face)) in_collision = 1;
        /* A position within `face` of an occupancy boundary: reported in
         * metres (the same grazing threshold applies). */
        if (face < edge) edge = face;
    }
    if (min_gap && edge < *min_gap) *min_gap = edge;
    return barrier + (in_collision ? P->c_obs : 0.0);
}

/* ------------------------------------------------------------------------
 * One rollout k (Alg. 1 inner loop, Eq. rollout_computation) and its cost
 * S_k = ComputeCost(x^k, u^k) (Eq. cost_1) with
 *   S_k = sum_{j=0..N} [rho_ref(x_j, x_ref_j) + obstacle(x_j)]
 *       + sum_{j=0..N-1} ||u_j||_R^2 + sum_{j=0..N-2} ||u_{j+1} - u_j||_Rd^2.
 * Reading (index ranges): u has N entries, so the input term runs over
 * j = 0..N-1 and the rate term over j = 0..N-2.  Reading: dynamics and
 * cost use the box-clamped control; the update uses the raw noise.
 * traj (optional) receives x_0..x_N, u_seq (optional) the clamped controls.
 * ---------------------------------------------------------------------- */
double orc_rollout(const orc_model* Mdl, const orc_params* P, const double x0[13],
                   const double* ref, const double* obs, int M, const double* u_nom,
                   uint64_t iter, uint32_t k, double* traj, double* u_seq, double* min_gap)
{
    int N = P->N;
    double x[13], x_next[13];
    memcpy(x, x0, sizeof(x));
    if (traj) memcpy(traj, x, sizeof(x));

    double S = orc_rho_ref(P, x, &ref[0]) + orc_obstacle_cost(P, x, obs, M, min_gap);
    double u_prev[4] = {0, 0, 0, 0};
    for (int j = 0; j < N; ++j) {
        double delta[4], u_raw[4], u[4];
        orc_noise(P, iter, k, (uint32_t)j, delta);
        for (int c = 0; c < 4; ++c) u_raw[c] = u_nom[4 * j + c] + delta[c];
        orc_clamp_input(Mdl, u_raw, u);
        if (u_seq) memcpy(&u_seq[4 * j], u, sizeof(u));

        S += orc_input_cost(P, u);
        if (j > 0) S += orc_rate_cost(P, u_prev, u);
        memcpy(u_prev, u, sizeof(u));

        double F_clip, tau_clip[3], w_clip[3];
        orc_feasible_input(Mdl, x, u, P->dt, &F_clip, tau_clip, w_clip);
        orc_rk4_step(Mdl, x, F_clip, tau_clip, P->dt, x_next);
        memcpy(x, x_next, sizeof(x));
        if (traj) memcpy(&traj[13 * (j + 1)], x, sizeof(x));

        S += orc_rho_ref(P, x, &ref[13 * (j + 1)]) + orc_obstacle_cost(P, x, obs, M, min_gap);
    }
    return S;
}

/* Weights of Eq. cost_2: rho = min S, w_k = exp(-(S_k - rho)/lambda)/eta.
 * Reading: a non-finite S_k gets weight 0; if every S_k is non-finite the
 * function returns ORC_ENONFINITE and leaves w untouched. */
int orc_weights(const double* S, int K, double lambda, double* w)
{
    double rho = INFINITY;
    for (int k = 0; k < K; ++k)
        if (isfinite(S[k]) && S[k] < rho) rho = S[k];
    if (!isfinite(rho)) return ORC_ENONFINITE;
    double eta = 0.0;
    for (int k = 0; k < K; ++k) eta += isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) : 0.0;
    for (int k = 0; k < K; ++k) w[k] = isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) / eta : 0.0;
    return ORC_OK;
}

/* Warm-start shift (Alg. 1, after ApplyToSystem): u_j <- u_{j+1},
 * u_{N-1} <- Initialize(u_{N-1}).  Reading: Initialize gives u_init
 * (hover) when tail_mode == 0 and keeps u_{N-1} when tail_mode == 1.
 * With 0 < alpha < 1 the nominal is resampled alpha steps later by linear
 * interpolation between knots instead (control-input interpolation,
 * Sec. IV-B); alpha == 1 is exactly the shift of Alg. 1. */
void orc_shift(const orc_params* P, const double* u, const double u_init[4], double* u_next)
{
    int N = P->N;
    double a = P->shift_alpha;
    for (int j = 0; j < N; ++j) {
        for (int c = 0; c < 4; ++c) {
            double later;
            if (j + 1 < N) later = u[4 * (j + 1) + c];
            else later = P->tail_mode == 1 ? u[4 * (N - 1) + c] : u_init[c];
            u_next[4 * j + c] = (1.0 - a) * u[4 * j + c] + a * later;
        }
    }
}

/* ------------------------------------------------------------------------
 * One MPPI iteration (Alg. 1, body of the while loop) for a given state
 * estimate x_hat, reference x_ref_0..x_ref_N, obstacle set and nominal
 * sequence u_nom (N x 4).  Outputs:
 *   u_out  (N x 4)  updated nominal, Eq. u_update (before the shift);
 *   u_cmd  (4)      [F_clip, omega_clip] from x_hat and u_out_0 (the
 *                   command sent to the low-level controller, Sec. III-B);
 *   u_next (N x 4)  warm start for the next iteration (shift / Sec. IV-B);
 *   x_next (13)     x_hat advanced by the applied command over the
 *                   control period alpha*dt (simulated plant, reading);
 *   costs  (K)      S_k; weights (K) w_k; min_gap (K) smallest distance of a
 *                   state's collision test from its boundary (test flag).
 * Any output pointer may be NULL.  Delay compensation (Sec. IV-E): with
 * delay > 0 the rollouts start from x_hat predicted forward by `delay`
 * seconds under the feasible input of u_nom_0.
 * Returns ORC_OK, ORC_EINVAL or ORC_ENONFINITE (then u_out = u_nom).
 * ---------------------------------------------------------------------- */
int orc_mppi_step(const orc_model* Mdl, const orc_params* P, const double x_hat[13],
                  const double* ref, const double* obs, int M, const double* u_nom,
                  uint64_t iter, int n_threads, double* u_out, double* u_cmd, double* u_next,
                  double* x_next, double* costs, double* weights, double* min_gap)
{
    int K = P->K, N = P->N;
    if (K < 1 || N < 1 || M < 0 || !(P->dt > 0.0) || !(P->lambda > 0.0)) return ORC_EINVAL;

    double x0[13];
    memcpy(x0, x_hat, sizeof(x0));
    if (P->delay > 0.0) {
        double u0[4], F, tau[3], wc[3];
        orc_clamp_input(Mdl, &u_nom[0], u0);
        orc_feasible_input(Mdl, x_hat, u0, P->dt, &F, tau, wc);
        orc_rk4_step(Mdl, x_hat, F, tau, P->delay, x0);
    }

    double* S = (double*)malloc(sizeof(double) * (size_t)K);
    double* w = (double*)malloc(sizeof(double) * (size_t)K);
    double* gaps = (double*)malloc(sizeof(double) * (size_t)K);
    if (!S || !w || !gaps) { free(S); free(w); free(gaps); return ORC_EINVAL; }

#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (int k = 0; k < K; ++k) {
        gaps[k] = INFINITY;
        S[k] = orc_rollout(Mdl, P, x0, ref, obs, M, u_nom, iter, (uint32_t)k, NULL, NULL, &gaps[k]);
    }
    (void)n_threads;

    int status = orc_weights(S, K, P->lambda, w);
    double* u_new = (double*)malloc(sizeof(double) * 4 * (size_t)N);
    if (status == ORC_OK) {
        /* Eq. u_update: u_nom_j := u_nom_j + sum_k w_k delta u_j^k. */
        for (int j = 0; j < N; ++j) {
            double acc[4] = {0, 0, 0, 0};
            for (int k = 0; k < K; ++k) {
                if (w[k] == 0.0) continue;
                double delta[4];
                orc_noise(P, iter, (uint32_t)k, (uint32_t)j, delta);
                for (int c = 0; c < 4; ++c) acc[c] += w[k] * delta[c];
            }
            for (int c = 0; c < 4; ++c) u_new[4 * j + c] = u_nom[4 * j + c] + acc[c];
        }
    } else {
        memcpy(u_new, u_nom, sizeof(double) * 4 * (size_t)N);
    }

    /* ApplyToSystem(u_nom_0): the feasible command from the current state. */
    double u0[4], F, tau[3], wc[3];
    double h_ctrl = P->shift_alpha * P->dt;
    orc_clamp_input(Mdl, &u_new[0], u0);
    orc_feasible_input(Mdl, x_hat, u0, P->dt, &F, tau, wc);
    if (u_cmd) { u_cmd[0] = F; u_cmd[1] = wc[0]; u_cmd[2] = wc[1]; u_cmd[3] = wc[2]; }
    if (x_next) orc_rk4_step(Mdl, x_hat, F, tau, h_ctrl, x_next);

    if (u_next) {
        double u_init[4] = {Mdl->mass * Mdl->g, 0.0, 0.0, 0.0};
        orc_shift(P, u_new, u_init, u_next);
    }
    if (u_out) memcpy(u_out, u_new, sizeof(double) * 4 * (size_t)N);
    if (costs) memcpy(costs, S, sizeof(double) * (size_t)K);
    if (weights) memcpy(weights, w, sizeof(double) * (size_t)K);
    if (min_gap) memcpy(min_gap, gaps, sizeof(double) * (size_t)K);
    free(S); free(w); free(gaps); free(u_new);
    return status;
}

/* Per-sample costs of a subset of rollouts (sampled parity at full size):
 * S_k for k in ks[0..n-1]. */
void orc_sample_costs(const orc_model* Mdl, const orc_params* P, const double x_hat[13],
                      const double* ref, const double* obs, int M, const double* u_nom,
                      uint64_t iter, const int* ks, int n, int n_threads, double* costs_out,
                      double* min_gap_out)
{
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
    for (int i = 0; i < n; ++i) {
        double g = INFINITY;
        costs_out[i] = orc_rollout(Mdl, P, x_hat, ref, obs, M, u_nom, iter, (uint32_t)ks[i], NULL,
                                   NULL, &g);
        if (min_gap_out) min_gap_out[i] = g;
    }
    (void)n_threads;
}

/* delta u_j^k for all (k, j): out[(k * N + j) * 4 + c] (test helper). */
void orc_noise_block(const orc_params* P, uint64_t iter, int K, int N, double* out)
{
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < N; ++j) orc_noise(P, iter, (uint32_t)k, (uint32_t)j, &out[(k * (size_t)N + j) * 4]);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
