// Solver service with continuous batching (not in the paper: the serving form of the
// hot path).  Requests (whole planning problems) are admitted in arrival order as soon as a
// slot is free and their device memory fits the budget; each admitted request runs the
// two-stage solve on its own non-blocking CUDA stream, so requests that arrive while others
// are on the GPU overlap with them on the device.  Host threads only orchestrate: all
// computation is the library's kernels.  Every host wait is bounded.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "spasm.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long ticket = 0;
    // deep copies of the inputs
    std::vector<double> dh, qlim, sphere, ee, q_home, cub, osph, half, init, box;
    std::vector<int32_t> link;
    spasm_robot robot{};
    spasm_obstacles obs{};
    spasm_goal goal{};
    spasm_params prm{};
    long long bytes = 0;
    int state = 0;   // 0 queued, 1 running, 2 done
    int status = SPASM_OK;
    std::string message;
    int n_found = 0;
    std::vector<double> placements, traj, cost;
    std::vector<int> success;
    Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct spasm_server {
    int device = 0;
    long long budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<long long, std::shared_ptr<Request>> all;
    std::vector<std::thread> workers;
    long long next_ticket = 1;
    bool stop = false;
};

// Device bytes a problem allocates (mirrors spasm_create_problem's allocations).
static long long problem_bytes(const spasm_obstacles* obs, const spasm_goal* goal, const spasm_params* p) {
    const long long B = goal->n_blocks, C = 2 * B * (p->W - 1) + 1, NR = 9 * B + 3;
    long long f = 0;
    f += 16LL * obs->n_cuboids + 4LL * obs->n_spheres;              // float tables
    f += 4 * B * (long long)p->N + p->N + 4 * B * (long long)p->M * 1 + 3LL * p->M + p->P + (long long)p->P * B * 4;
    f += (long long)p->Q * C * 8 + (long long)p->Q * NR + p->Q + 8LL * p->Q + 2LL * p->Q + (long long)p->P * C * 8;
    f += 64;
    long long d = 16LL * obs->n_cuboids + 4LL * obs->n_spheres + 6LL * p->P;   // double tables
    return 4 * f + 8 * d + (1 << 16);
}

static void run_request(spasm_server* sv, Request& r, cudaStream_t st) {
    spasm_problem_t pr = nullptr;
    int status = spasm_create_problem(&r.robot, &r.obs, &r.goal, &r.prm, st, &pr);
    if (status == SPASM_OK) status = spasm_optimize(pr);
    if (status == SPASM_OK || status == SPASM_ERR_NOSOLUTION) {
        const int P = r.prm.P, B = r.goal.n_blocks, C = 2 * B * (r.prm.W - 1) + 1;
        r.placements.assign((size_t)P * B * 4, 0.0);
        r.traj.assign((size_t)P * C * 7, 0.0);
        r.cost.assign(P, 0.0);
        r.success.assign(P, 0);
        int nf = 0;
        const int st2 = spasm_result(pr, &nf, r.placements.data(), r.traj.data(), r.cost.data(), r.success.data());
        if (st2 != SPASM_OK && st2 != SPASM_ERR_NOSOLUTION) status = st2;
        r.n_found = nf;
    }
    if (status != SPASM_OK) r.message = spasm_last_error();
    if (pr) spasm_destroy_problem(pr);
    cudaStreamSynchronize(st);
    (void)sv;
    r.status = status;
}

static void worker_loop(spasm_server* sv) {
    cudaSetDevice(sv->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // admit the oldest request once its memory fits (a request larger than the whole
            // budget runs alone)
            sv->cv_work.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->queue.empty()) return false;
                const long long need = sv->queue.front()->bytes;
                return sv->in_use + need <= sv->budget || sv->in_use == 0;
            });
            if (sv->stop && sv->queue.empty()) break;
            if (sv->queue.empty()) continue;
            r = sv->queue.front();
            sv->queue.pop_front();
            sv->in_use += r->bytes;
            r->state = 1;
            r->t_start = Clock::now();
        }
        run_request(sv, *r, st);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->in_use -= r->bytes;
            r->t_done = Clock::now();
            r->state = 2;
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    cudaStreamDestroy(st);
}

extern "C" spasm_status spasm_server_create(long long budget_bytes, int max_inflight, spasm_server_t* out) {
    if (!out || budget_bytes <= 0 || max_inflight < 1 || max_inflight > 256) return SPASM_ERR_INVALID;
    auto* sv = new spasm_server();
    cudaGetDevice(&sv->device);
    sv->budget = budget_bytes;
    for (int i = 0; i < max_inflight; ++i) sv->workers.emplace_back(worker_loop, sv);
    *out = sv;
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_submit(spasm_server_t sv, const spasm_robot* robot, const spasm_obstacles* obs,
                                            const spasm_goal* goal, const spasm_params* prm, long long* ticket) {
    if (!sv || !robot || !obs || !goal || !prm || !ticket) return SPASM_ERR_INVALID;
    if (robot->dof != 7 || goal->n_blocks < 1 || goal->n_blocks > spasm::kMaxB || prm->W < 3 ||
        robot->n_spheres < 1 || robot->n_spheres > spasm::kMaxRobotSpheres || obs->n_cuboids < 0 ||
        obs->n_cuboids > spasm::kMaxCub || obs->n_spheres < 0 || obs->n_spheres > spasm::kMaxOSph)
        return SPASM_ERR_INVALID;
    auto r = std::make_shared<Request>();
    const int B = goal->n_blocks, ns = robot->n_spheres;
    r->dh.assign(robot->dh, robot->dh + 28);
    r->qlim.assign(robot->qlim, robot->qlim + 14);
    r->sphere.assign(robot->sphere, robot->sphere + 4 * ns);
    r->link.assign(robot->sphere_link, robot->sphere_link + ns);
    r->ee.assign(robot->ee, robot->ee + 16);
    r->q_home.assign(robot->q_home, robot->q_home + 7);
    r->cub.assign(obs->cuboid, obs->cuboid + 15 * obs->n_cuboids);
    r->osph.assign(obs->sphere, obs->sphere + 4 * obs->n_spheres);
    r->half.assign(goal->half_ext, goal->half_ext + 3 * B);
    r->init.assign(goal->init_pose, goal->init_pose + 4 * B);
    r->box.assign(goal->goal_box, goal->goal_box + 6);
    r->robot = *robot;
    r->robot.dh = r->dh.data(); r->robot.qlim = r->qlim.data(); r->robot.sphere = r->sphere.data();
    r->robot.sphere_link = r->link.data(); r->robot.ee = r->ee.data(); r->robot.q_home = r->q_home.data();
    r->obs = *obs;
    r->obs.cuboid = r->cub.data(); r->obs.sphere = r->osph.data();
    r->goal = *goal;
    r->goal.half_ext = r->half.data(); r->goal.init_pose = r->init.data(); r->goal.goal_box = r->box.data();
    r->prm = *prm;
    r->bytes = problem_bytes(obs, goal, prm);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->ticket = sv->next_ticket++;
        sv->queue.push_back(r);
        sv->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    sv->cv_work.notify_all();
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_poll(spasm_server_t sv, long long ticket, int* state) {
    if (!sv || !state) return SPASM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return SPASM_ERR_INVALID;
    *state = it->second->state;
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_wait(spasm_server_t sv, long long ticket, double timeout_s) {
    if (!sv) return SPASM_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return SPASM_ERR_INVALID;
    auto r = it->second;
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->state == 2; });
    return ok ? SPASM_OK : SPASM_ERR_TIMEOUT;
}

extern "C" spasm_status spasm_server_result(spasm_server_t sv, long long ticket, int* status, int* n_found,
                                            double* placements, double* traj, double* cost, int* success,
                                            double* latency_ms, double* queue_ms) {
    if (!sv) return SPASM_ERR_INVALID;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(ticket);
        if (it == sv->all.end()) return SPASM_ERR_INVALID;
        r = it->second;
        if (r->state != 2) return SPASM_ERR_TIMEOUT;
    }
    if (status) *status = r->status;
    if (n_found) *n_found = r->n_found;
    if (placements && !r->placements.empty()) std::memcpy(placements, r->placements.data(), r->placements.size() * 8);
    if (traj && !r->traj.empty()) std::memcpy(traj, r->traj.data(), r->traj.size() * 8);
    if (cost && !r->cost.empty()) std::memcpy(cost, r->cost.data(), r->cost.size() * 8);
    if (success && !r->success.empty()) std::memcpy(success, r->success.data(), r->success.size() * sizeof(int));
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (queue_ms) *queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_release(spasm_server_t sv, long long ticket) {
    if (!sv) return SPASM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return SPASM_ERR_INVALID;
    if (it->second->state != 2) return SPASM_ERR_INVALID;
    sv->all.erase(it);
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_destroy(spasm_server_t sv) {
    if (!sv) return SPASM_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
    return SPASM_OK;
}
