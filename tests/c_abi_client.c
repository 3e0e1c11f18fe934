/* A plain C99 client of include/mppi.h, built and run by the tests.
 *
 *   c_abi_client layout
 *       prints "struct field offset size" for every field of every public
 *       struct and "struct - 0 sizeof" for the struct itself, so that the
 *       Python binding's mirrors can be checked against the C layout;
 *   c_abi_client solve IN OUT
 *       IN holds int32 M, then the bytes of an mppi_model and an
 *       mppi_params, then x_hat[13], ref[(N+1)*13], obstacles[M*4],
 *       u_nom[N*4] (float32) and uint64 iter; one mppi_solve with host
 *       buffers; OUT receives int32 status, u_out[N*4], u_cmd[4],
 *       u_next[N*4], x_next[13].
 */
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

#include "mppi.h"

#define F(S, f) printf(#S " " #f " %zu %zu\n", offsetof(S, f), sizeof(((S*)0)->f))
#define S(S) printf(#S " - 0 %zu\n", sizeof(S))

static void layout(void) {
    S(mppi_model);
    F(mppi_model, mass); F(mppi_model, g); F(mppi_model, arm_l); F(mppi_model, c_tf); F(mppi_model, J);
    F(mppi_model, T_min); F(mppi_model, T_max); F(mppi_model, motor_clip); F(mppi_model, F_min);
    F(mppi_model, F_max); F(mppi_model, w_max);
    S(mppi_params);
    F(mppi_params, K); F(mppi_params, N); F(mppi_params, dt); F(mppi_params, lambda); F(mppi_params, sigma);
    F(mppi_params, c_p); F(mppi_params, c_q); F(mppi_params, c_v); F(mppi_params, c_w); F(mppi_params, R);
    F(mppi_params, Rd); F(mppi_params, c_obs); F(mppi_params, c_bar); F(mppi_params, beta);
    F(mppi_params, r_uav); F(mppi_params, quat_metric); F(mppi_params, tail_mode); F(mppi_params, shift_alpha);
    F(mppi_params, delay); F(mppi_params, seed); F(mppi_params, stream_id); F(mppi_params, reserved);
    S(mppi_capacity);
    F(mppi_capacity, max_instances); F(mppi_capacity, max_samples); F(mppi_capacity, N_max);
    F(mppi_capacity, M_max);
    S(mppi_instance);
    F(mppi_instance, x_hat); F(mppi_instance, ref); F(mppi_instance, obstacles); F(mppi_instance, u_nom);
    F(mppi_instance, u_out); F(mppi_instance, u_cmd); F(mppi_instance, u_next); F(mppi_instance, x_next);
    F(mppi_instance, costs); F(mppi_instance, status); F(mppi_instance, iter_dev); F(mppi_instance, iter);
    F(mppi_instance, K); F(mppi_instance, N); F(mppi_instance, M); F(mppi_instance, dt);
    F(mppi_instance, lambda); F(mppi_instance, sigma); F(mppi_instance, seed); F(mppi_instance, stream_id);
    F(mppi_instance, reserved);
    S(mppi_shape);
    F(mppi_shape, block); F(mppi_shape, lanes); F(mppi_shape, pipelined); F(mppi_shape, list_margin);
    F(mppi_shape, samples_per_thread);
    S(mppi_server_cfg);
    F(mppi_server_cfg, max_vehicles); F(mppi_server_cfg, slots); F(mppi_server_cfg, max_batch);
    F(mppi_server_cfg, N_max); F(mppi_server_cfg, M_max); F(mppi_server_cfg, queue_capacity);
    F(mppi_server_cfg, max_batch_samples); F(mppi_server_cfg, hbm_budget_bytes); F(mppi_server_cfg, block);
    F(mppi_server_cfg, lanes);
    S(mppi_result);
    F(mppi_result, request_id); F(mppi_result, vehicle); F(mppi_result, status); F(mppi_result, u_cmd);
    F(mppi_result, u0); F(mppi_result, t_submit_us); F(mppi_result, t_done_us); F(mppi_result, batch_size);
    F(mppi_result, reserved);
    S(mppi_server_stats);
    F(mppi_server_stats, submitted); F(mppi_server_stats, completed); F(mppi_server_stats, rejected);
    F(mppi_server_stats, batches); F(mppi_server_stats, instances); F(mppi_server_stats, bytes_in_use);
    F(mppi_server_stats, bytes_budget); F(mppi_server_stats, busy_us);
    S(mppi_peaks);
    F(mppi_peaks, sm_count); F(mppi_peaks, reserved); F(mppi_peaks, fp32_flops); F(mppi_peaks, fp32_ms);
    F(mppi_peaks, ex2_ops); F(mppi_peaks, lg2_ops); F(mppi_peaks, rsqrt_ops); F(mppi_peaks, sin_ops);
    F(mppi_peaks, cos_ops);
}

static int read_all(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n; }

static int solve(const char* in_path, const char* out_path) {
    FILE* f = fopen(in_path, "rb");
    if (!f) return 2;
    int32_t M;
    mppi_model model;
    mppi_params params;
    int ok = read_all(f, &M, sizeof M) && read_all(f, &model, sizeof model) && read_all(f, &params, sizeof params);
    if (!ok || M < 0 || params.N < 1) {
        fclose(f);
        return 2;
    }
    const size_t N = (size_t)params.N;
    float* x_hat = malloc(13 * sizeof(float));
    float* ref = malloc(13 * (N + 1) * sizeof(float));
    float* obs = malloc((4 * (size_t)M + 1) * sizeof(float));
    float* u_nom = malloc(4 * N * sizeof(float));
    float* u_out = malloc(4 * N * sizeof(float));
    float* u_next = malloc(4 * N * sizeof(float));
    float u_cmd[4], x_next[13];
    uint64_t iter = 0;
    ok = x_hat && ref && obs && u_nom && u_out && u_next && read_all(f, x_hat, 13 * sizeof(float)) &&
         read_all(f, ref, 13 * (N + 1) * sizeof(float)) && read_all(f, obs, 4 * (size_t)M * sizeof(float)) &&
         read_all(f, u_nom, 4 * N * sizeof(float)) && read_all(f, &iter, sizeof iter);
    fclose(f);
    int32_t status = -100;
    if (ok) {
        mppi_handle h = NULL;
        status = mppi_create(&model, &params, NULL, &h);
        if (status == MPPI_OK) {
            status = mppi_solve(h, x_hat, ref, M > 0 ? obs : NULL, M, u_nom, iter, u_out, u_cmd, u_next, x_next,
                                NULL);
            mppi_destroy(h);
        } else {
            fprintf(stderr, "mppi_create: %s\n", mppi_strerror(status));
        }
    }
    FILE* o = fopen(out_path, "wb");
    if (o) {
        fwrite(&status, sizeof status, 1, o);
        fwrite(u_out, sizeof(float), 4 * N, o);
        fwrite(u_cmd, sizeof(float), 4, o);
        fwrite(u_next, sizeof(float), 4 * N, o);
        fwrite(x_next, sizeof(float), 13, o);
        fclose(o);
    }
    free(x_hat); free(ref); free(obs); free(u_nom); free(u_out); free(u_next);
    return ok && o ? 0 : 2;
}

int main(int argc, char** argv) {
    if (argc == 2 && argv[1][0] == 'l') {
        layout();
        return 0;
    }
    if (argc == 4) return solve(argv[2], argv[3]);
    fprintf(stderr, "usage: %s layout | solve IN OUT\n", argv[0]);
    return 2;
}
