// Serving runtime: continuous batching of MPPI solve requests from many
// vehicles on one GPU.
//
// Vehicles keep their warm-start nominal sequence and Philox counter in
// device memory; a request carries only the state estimate and the
// reference window.  One dispatcher thread owns the GPU work: whenever a
// launch slot (a handle with its own workspace, graph cache and stream) is
// free and requests are queued, it takes queued requests of vehicles that
// have nothing in flight (in arrival order, up to the slot's instance and
// sample limits), copies their inputs into the slot's pinned staging,
// replays the batched kernel from the slot's CUDA graph and records an
// event.  Slots run concurrently, so requests arriving while earlier
// batches are on the GPU join the next free slot and their work overlaps.
// Completed slots are detected by event queries; results go to a completion
// queue the client polls.  Device memory is admitted against a budget:
// slot workspaces are reserved at creation, each vehicle's state when it is
// added.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mppi_internal.h"

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Vehicle {
    bool live = false;
    int K = 0, N = 0, M = 0;
    float dt = 0, lambda = 0, sigma[4] = {0, 0, 0, 0};
    uint64_t seed = 0;
    uint32_t stream_id = 0;
    float* d_obs = nullptr;
    float* d_unom = nullptr;
    unsigned long long* d_iter = nullptr;
    size_t bytes = 0;
    int in_flight = 0;   // requests dispatched and not completed (0 or 1)
    int queued = 0;      // requests waiting in the queue
    bool removing = false;  // being removed: its pending requests finish, no new ones
};

struct Request {
    uint64_t id;
    int vid;
    double t_submit;
    std::vector<float> in;  // x_hat (16 floats, padded) + ref ((N+1)*13)
};

// Per-instance result block in a slot's output buffer (floats):
// u_cmd[4], status (int32 bits), 3 pad, then u_out[N_max][4].
constexpr int kOutHead = 8;

struct Slot {
    mppi_handle h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float* h_in = nullptr;
    float* d_in = nullptr;
    size_t in_floats = 0;
    float* h_out = nullptr;
    float* d_out = nullptr;      // [max_batch][kOutHead + 4 N_max]
    size_t out_stride = 0;
    std::vector<Request> batch;
    std::vector<mppi_instance> desc;
    bool busy = false;
    double t_launch = 0;
};

}  // namespace

struct mppi_server {
    mppi_model model{};
    mppi_params params{};
    mppi_server_cfg cfg{};
    int device = 0;

    std::mutex mu;
    std::condition_variable cv;       // submit / drain wake-ups
    std::condition_variable cv_done;  // completions
    std::deque<Request> queue;
    std::deque<mppi_result> completed;
    std::vector<Vehicle> vehicles;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int in_flight = 0;

    int64_t bytes_reserved = 0;  // slot workspaces and staging
    int64_t bytes_vehicles = 0;
    mppi_server_stats stats{};
};

namespace {

// Device bytes one slot may use: the handle's tile partials for the worst
// launch shape (8 samples per tile), counters, descriptors, staging.
int64_t slot_bytes(const mppi_server_cfg& c) {
    const int64_t tiles = c.max_batch_samples / 8 + c.max_batch;
    const int64_t partials = tiles * (4 + 4 * (int64_t)c.N_max) * 4;
    const int64_t staging = (int64_t)c.max_batch * (16 + 13 * (int64_t)(c.N_max + 1)) * 4;
    const int64_t outs = (int64_t)c.max_batch * (kOutHead + 4 * (int64_t)c.N_max) * 4;
    const int64_t desc = (int64_t)c.max_batch * (256 + 8) + tiles * 8 + 4096;
    return partials + staging + outs + desc;
}

int64_t vehicle_bytes(int N, int M) {
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    return up(16 * (int64_t)M) + up(16 * (int64_t)N) + up(8);
}

void free_vehicle(Vehicle& v) {
    cudaFree(v.d_obs);
    cudaFree(v.d_unom);
    cudaFree(v.d_iter);
    v = Vehicle();
}

// Takes requests for a free slot (caller holds the lock).
void pick_batch(mppi_server* s, Slot& slot) {
    slot.batch.clear();
    int64_t samples = 0;
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)slot.batch.size() < s->cfg.max_batch;) {
        Vehicle& v = s->vehicles[it->vid];
        if (v.in_flight > 0 || samples + v.K > s->cfg.max_batch_samples) {
            ++it;
            continue;
        }
        samples += v.K;
        v.in_flight = 1;
        v.queued -= 1;
        slot.batch.push_back(std::move(*it));
        it = s->queue.erase(it);
    }
}

// Stages and launches a slot's batch (lock not held).
int launch_slot(mppi_server* s, Slot& slot) {
    const int n = (int)slot.batch.size();
    size_t off = 0;
    slot.desc.resize(n);
    for (int i = 0; i < n; ++i) {
        const Request& r = slot.batch[i];
        const Vehicle& v = s->vehicles[r.vid];
        std::memcpy(slot.h_in + off, r.in.data(), r.in.size() * sizeof(float));
        mppi_instance& d = slot.desc[i];
        std::memset(&d, 0, sizeof(d));
        d.x_hat = slot.d_in + off;
        d.ref = slot.d_in + off + 16;
        d.obstacles = v.M > 0 ? v.d_obs : nullptr;
        d.u_nom = v.d_unom;
        d.u_next = v.d_unom;  // warm start replaced in place
        float* o = slot.d_out + (size_t)i * slot.out_stride;
        d.u_cmd = o;
        d.status = reinterpret_cast<int32_t*>(o + 4);
        d.u_out = o + kOutHead;
        d.iter_dev = reinterpret_cast<uint64_t*>(v.d_iter);
        d.K = v.K; d.N = v.N; d.M = v.M;
        d.dt = v.dt; d.lambda = v.lambda;
        for (int c = 0; c < 4; ++c) d.sigma[c] = v.sigma[c];
        d.seed = v.seed;
        d.stream_id = v.stream_id;
        off += (r.in.size() + 3) / 4 * 4;
    }
    cudaStream_t st = slot.stream;
    if (cudaMemcpyAsync(slot.d_in, slot.h_in, off * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MPPI_ECUDA;
    int rc = mppi_solve_batch_graph(slot.h, slot.desc.data(), n, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(slot.h_out, slot.d_out, (size_t)n * slot.out_stride * sizeof(float), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaEventRecord(slot.done, st) != cudaSuccess)
        return MPPI_ECUDA;
    return MPPI_OK;
}

// Collects a finished slot's results (caller holds the lock).
void finish_slot(mppi_server* s, Slot& slot, int launch_rc) {
    const double t = now_us();
    const int n = (int)slot.batch.size();
    for (int i = 0; i < n; ++i) {
        const Request& r = slot.batch[i];
        mppi_result res;
        std::memset(&res, 0, sizeof(res));
        res.request_id = r.id;
        res.vehicle = r.vid;
        const float* o = slot.h_out + (size_t)i * slot.out_stride;
        int32_t st = 0;
        std::memcpy(&st, o + 4, sizeof(st));
        res.status = launch_rc ? launch_rc : st;
        if (!launch_rc) {
            std::memcpy(res.u_cmd, o, 4 * sizeof(float));
            std::memcpy(res.u0, o + kOutHead, 4 * sizeof(float));
        }
        res.t_submit_us = r.t_submit;
        res.t_done_us = t;
        res.batch_size = n;
        s->completed.push_back(res);
        s->vehicles[r.vid].in_flight = 0;
    }
    s->stats.completed += n;
    s->stats.batches += 1;
    s->stats.instances += n;
    s->stats.busy_us += t - slot.t_launch;
    s->in_flight -= n;
    slot.batch.clear();
    slot.busy = false;
}

void dispatcher(mppi_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        for (Slot& slot : s->slots) {
            if (!slot.busy) continue;
            lk.unlock();
            const cudaError_t q = cudaEventQuery(slot.done);
            lk.lock();
            if (q == cudaErrorNotReady) continue;
            finish_slot(s, slot, q == cudaSuccess ? MPPI_OK : MPPI_ECUDA);
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        for (Slot& slot : s->slots) {
            if (slot.busy || s->queue.empty()) continue;
            pick_batch(s, slot);
            if (slot.batch.empty()) continue;
            slot.busy = true;
            slot.t_launch = now_us();
            lk.unlock();
            const int rc = launch_slot(s, slot);
            if (rc) {
                // Copies enqueued before the failure may still read the
                // slot's staging; the slot is reused only after they end.
                cudaStreamSynchronize(slot.stream);
                cudaGetLastError();
            }
            lk.lock();
            if (rc) {
                finish_slot(s, slot, rc);
                s->cv_done.notify_all();
            }
            progressed = true;
        }
        if (s->stop && s->queue.empty() && s->in_flight == 0) break;
        if (!progressed) {
            bool any_busy = false;
            for (Slot& slot : s->slots) any_busy |= slot.busy;
            if (any_busy) {
                // Batches in flight: poll their events again at once (the
                // dispatcher owns one host core; a timed sleep would add the
                // timer's slack, tens of microseconds, to every completion).
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
}

void destroy_slots(mppi_server* s) {
    for (Slot& slot : s->slots) {
        if (slot.stream) cudaStreamSynchronize(slot.stream);
        if (slot.h) mppi_destroy(slot.h);
        if (slot.done) cudaEventDestroy(slot.done);
        if (slot.stream) cudaStreamDestroy(slot.stream);
        if (slot.h_in) cudaFreeHost(slot.h_in);
        if (slot.h_out) cudaFreeHost(slot.h_out);
        cudaFree(slot.d_in);
        cudaFree(slot.d_out);
    }
    s->slots.clear();
}

// A live vehicle that is not being removed, or NULL.
Vehicle* find_vehicle(mppi_server* s, int vid) {
    if (vid < 0 || vid >= (int)s->vehicles.size() || !s->vehicles[vid].live || s->vehicles[vid].removing)
        return nullptr;
    return &s->vehicles[vid];
}

}  // namespace

extern "C" {

int mppi_server_create(const mppi_model* model, const mppi_params* params, const mppi_server_cfg* cfg,
                       mppi_server** out) {
    if (!out || !cfg) return MPPI_EINVAL;
    *out = nullptr;
    int rc = mppi::check_model(model);
    if (rc) return rc;
    if ((rc = mppi::check_params(params))) return rc;
    const mppi_server_cfg& c = *cfg;
    if (c.max_vehicles < 1 || c.slots < 1 || c.slots > 64 || c.max_batch < 1 || c.N_max < 1 ||
        c.N_max > MPPI_N_MAX || c.M_max < 0 || c.M_max > MPPI_M_MAX || c.queue_capacity < 1 ||
        c.max_batch_samples < 1 || c.hbm_budget_bytes < 1)
        return MPPI_EINVAL;
    if ((c.block || c.lanes) && !mppi::shape_supported(mppi::Shape{c.block, c.lanes, 0})) return MPPI_EINVAL;
    const int64_t reserve = (int64_t)c.slots * slot_bytes(c);
    if (reserve > c.hbm_budget_bytes) return MPPI_ENOMEM;

    mppi_server* s = new (std::nothrow) mppi_server();
    if (!s) return MPPI_ENOMEM;
    s->model = *model;
    s->params = *params;
    s->cfg = c;
    cudaGetDevice(&s->device);
    s->vehicles.resize(c.max_vehicles);
    s->bytes_reserved = reserve;
    s->slots.resize(c.slots);
    const size_t in_floats = (size_t)c.max_batch * (16 + (13 * (size_t)(c.N_max + 1) + 3) / 4 * 4);
    for (Slot& slot : s->slots) {
        mppi_capacity cap;
        cap.max_instances = c.max_batch;
        cap.max_samples = c.max_batch_samples;
        cap.N_max = c.N_max;
        cap.M_max = c.M_max;
        mppi_params p = *params;
        p.K = (int)std::min<int64_t>(c.max_batch_samples, MPPI_K_MAX);
        p.N = c.N_max;
        if ((rc = mppi_create(model, &p, &cap, &slot.h))) break;
        if (c.block || c.lanes) {
            mppi_shape sh{c.block, c.lanes, 0};
            mppi_set_shape(slot.h, &sh);
        }
        slot.in_floats = in_floats;
        slot.out_stride = kOutHead + 4 * (size_t)c.N_max;
        if (cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&slot.h_in, in_floats * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&slot.d_in, in_floats * sizeof(float)) != cudaSuccess ||
            cudaMallocHost(&slot.h_out, (size_t)c.max_batch * slot.out_stride * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&slot.d_out, (size_t)c.max_batch * slot.out_stride * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            rc = MPPI_ENOMEM;
            break;
        }
    }
    if (rc) {
        destroy_slots(s);
        delete s;
        return rc;
    }
    s->stats.bytes_budget = c.hbm_budget_bytes;
    s->stats.bytes_in_use = reserve;
    s->worker = std::thread(dispatcher, s);
    *out = s;
    return MPPI_OK;
}

int mppi_server_add_vehicle(mppi_server* s, int32_t K, int32_t N, float dt, float lambda, const float* sigma,
                            const float* obstacles, int32_t M, const float* u_init, uint64_t seed,
                            uint32_t stream_id, int32_t* vehicle_id) {
    if (!s || !sigma || !vehicle_id) return MPPI_EINVAL;
    if (mppi::check_step(K, N, dt, lambda, sigma)) return MPPI_EINVAL;
    if (N > s->cfg.N_max || M < 0 || M > s->cfg.M_max || K > s->cfg.max_batch_samples) return MPPI_EINVAL;
    if (M > 0 && !obstacles) return MPPI_EINVAL;
    const int64_t need = vehicle_bytes(N, M);
    std::unique_lock<std::mutex> lk(s->mu);
    int vid = -1;
    for (int i = 0; i < (int)s->vehicles.size(); ++i)
        if (!s->vehicles[i].live) {
            vid = i;
            break;
        }
    if (vid < 0) return MPPI_ENOMEM;
    if (s->bytes_reserved + s->bytes_vehicles + need > s->cfg.hbm_budget_bytes) return MPPI_ENOMEM;
    Vehicle v;
    v.K = K; v.N = N; v.M = M; v.dt = dt; v.lambda = lambda;
    for (int c = 0; c < 4; ++c) v.sigma[c] = sigma[c];
    v.seed = seed;
    v.stream_id = stream_id;
    v.bytes = (size_t)need;
    std::vector<float> u0(4 * (size_t)N, 0.0f);
    if (u_init) std::memcpy(u0.data(), u_init, u0.size() * sizeof(float));
    else
        for (int j = 0; j < N; ++j) u0[4 * (size_t)j] = s->model.mass * s->model.g;
    const unsigned long long zero = 0;
    if ((M > 0 && cudaMalloc(&v.d_obs, 16 * (size_t)M) != cudaSuccess) ||
        cudaMalloc(&v.d_unom, 16 * (size_t)N) != cudaSuccess || cudaMalloc(&v.d_iter, 8) != cudaSuccess ||
        (M > 0 && cudaMemcpy(v.d_obs, obstacles, 16 * (size_t)M, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(v.d_unom, u0.data(), 16 * (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v.d_iter, &zero, 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        free_vehicle(v);
        return MPPI_ENOMEM;
    }
    v.live = true;
    s->vehicles[vid] = v;
    s->bytes_vehicles += need;
    s->stats.bytes_in_use = s->bytes_reserved + s->bytes_vehicles;
    *vehicle_id = vid;
    return MPPI_OK;
}

int mppi_server_remove_vehicle(mppi_server* s, int32_t vid) {
    if (!s) return MPPI_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    Vehicle* v = find_vehicle(s, vid);
    if (!v) return MPPI_ENOTFOUND;
    // From here on the vehicle takes no new request and a second removal
    // finds nothing; the requests already queued or in flight complete.
    v->removing = true;
    s->cv_done.wait(lk, [&] { return v->in_flight == 0 && v->queued == 0; });
    s->bytes_vehicles -= (int64_t)v->bytes;
    s->stats.bytes_in_use = s->bytes_reserved + s->bytes_vehicles;
    free_vehicle(*v);
    return MPPI_OK;
}

int mppi_server_submit(mppi_server* s, int32_t vid, const float* x_hat, const float* ref, uint64_t* request_id) {
    if (!s || !x_hat || !ref) return MPPI_EINVAL;
    Request r;
    std::unique_lock<std::mutex> lk(s->mu);
    Vehicle* v = find_vehicle(s, vid);
    if (!v) return MPPI_ENOTFOUND;
    if ((int)s->queue.size() >= s->cfg.queue_capacity) {
        s->stats.rejected += 1;
        return MPPI_EAGAIN;
    }
    const size_t nref = 13 * (size_t)(v->N + 1);
    r.in.assign(16 + nref, 0.0f);
    std::memcpy(r.in.data(), x_hat, 13 * sizeof(float));
    std::memcpy(r.in.data() + 16, ref, nref * sizeof(float));
    r.vid = vid;
    r.id = s->next_id++;
    r.t_submit = now_us();
    if (request_id) *request_id = r.id;
    v->queued += 1;
    s->in_flight += 1;
    s->stats.submitted += 1;
    s->queue.push_back(std::move(r));
    lk.unlock();
    s->cv.notify_one();
    return MPPI_OK;
}

int mppi_server_poll(mppi_server* s, mppi_result* out, int32_t max, int32_t* n) {
    if (!s || !n || max < 0 || (max > 0 && !out)) return MPPI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    int k = 0;
    while (k < max && !s->completed.empty()) {
        out[k++] = s->completed.front();
        s->completed.pop_front();
    }
    *n = k;
    return MPPI_OK;
}

int mppi_server_drain(mppi_server* s, int32_t timeout_ms) {
    if (!s) return MPPI_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->in_flight == 0; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, idle);
        return MPPI_OK;
    }
    return s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle) ? MPPI_OK : MPPI_ETIMEOUT;
}

int mppi_server_export_vehicle(mppi_server* s, int32_t vid, float* u_nom, uint64_t* iter) {
    if (!s || !u_nom || !iter) return MPPI_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    Vehicle* v = find_vehicle(s, vid);
    if (!v) return MPPI_ENOTFOUND;
    s->cv_done.wait(lk, [&] { return v->in_flight == 0; });
    if (!v->live || v->removing) return MPPI_ENOTFOUND;  // removed while waiting
    unsigned long long it = 0;
    if (cudaMemcpy(u_nom, v->d_unom, 16 * (size_t)v->N, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&it, v->d_iter, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return MPPI_ECUDA;
    *iter = it;
    return MPPI_OK;
}

int mppi_server_import_vehicle(mppi_server* s, int32_t vid, const float* u_nom, uint64_t iter) {
    if (!s || !u_nom) return MPPI_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    Vehicle* v = find_vehicle(s, vid);
    if (!v) return MPPI_ENOTFOUND;
    s->cv_done.wait(lk, [&] { return v->in_flight == 0; });
    if (!v->live || v->removing) return MPPI_ENOTFOUND;  // removed while waiting
    const unsigned long long it = iter;
    if (cudaMemcpy(v->d_unom, u_nom, 16 * (size_t)v->N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v->d_iter, &it, 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return MPPI_ECUDA;
    return MPPI_OK;
}

int mppi_server_get_stats(mppi_server* s, mppi_server_stats* st) {
    if (!s || !st) return MPPI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    return MPPI_OK;
}

int mppi_server_destroy(mppi_server* s) {
    if (!s) return MPPI_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    destroy_slots(s);
    for (Vehicle& v : s->vehicles)
        if (v.live) free_vehicle(v);
    delete s;
    return MPPI_OK;
}

}  // extern "C"
