// Solver service with continuous batching (not in the paper: the serving form of the hot path).
//
// One scheduler thread owns the device work.  It runs in epochs; each epoch is one trajectory
// attempt of every request in flight, batched:
//   1. admit queued requests in arrival order while a slot is free and their device memory
//      (spasm_problem_bytes, the allocation list of spasm_create_problem) fits the budget; a
//      request larger than the whole budget is admitted when nothing else is in flight;
//   2. create each admitted request's problem and enqueue its stage 1 (the graph with the
//      device-side attempt loop of spasm_place) and its first lift;
//   3. one persistent launch of the trajectory kernel over the particles of every request in
//      flight (a shared work list of particle runs, gated per request by its placement count);
//   4. per request: the satisfying selection and the attempt decision on the device, and the
//      FP64 check of the best P;
//   5. one host wait, then retire the requests that finished (results copied to the host,
//      problems destroyed, budget returned) and re-lift the others with their next attempt
//      counter for the next epoch.
// Requests that arrive during an epoch join at the next one, so the GPU runs one launch over
// all work in flight rather than one solve per request.  Every particle runs the code of a
// single solve with the same Philox streams, so a request's result does not depend on what
// else is in flight.  Host waits are bounded; a request is cancelled while it is queued, or
// at the next epoch boundary while it is in flight.
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

#include "problem.h"

using namespace spasm;

namespace {

using Clock = std::chrono::steady_clock;

enum { kQueued = 0, kRunning = 1, kDone = 2, kCancelled = 3 };

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
    int state = kQueued;
    bool cancel = false;
    int status = SPASM_OK;
    std::string message;
    int n_found = 0;
    std::vector<double> placements, traj, cost;
    std::vector<int> success;
    Clock::time_point t_submit, t_start, t_done;
    // scheduler-thread state
    spasm_problem_t pr = nullptr;
    int epochs = 0;
};

}  // namespace

struct spasm_server {
    int device = 0;
    long long budget = 0, in_use = 0;
    int max_inflight = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<long long, std::shared_ptr<Request>> all;
    std::thread scheduler;
    long long next_ticket = 1;
    bool stop = false;
    spasm_server_stats stats{};
};

namespace {

void finish_request(spasm_server* sv, Request& r, int status, const std::string& msg) {
    if (r.pr) {
        spasm_destroy_problem(r.pr);
        r.pr = nullptr;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r.cancel) {
        r.state = kCancelled;
        r.status = SPASM_ERR_CANCELLED;
        r.message = "cancelled";
    } else {
        r.state = kDone;
        r.status = status;
        r.message = msg;
    }
    sv->in_use -= r.bytes;
    r.t_done = Clock::now();
    sv->stats.completed += 1;
}

// Outputs of a finished request, read through the problem's own result call.
int read_result(Request& r) {
    const int P = r.prm.P, B = r.goal.n_blocks, C = 2 * B * (r.prm.W - 1) + 1;
    r.placements.assign((size_t)P * B * 4, 0.0);
    r.traj.assign((size_t)P * C * 7, 0.0);
    r.cost.assign(P, 0.0);
    r.success.assign(P, 0);
    int nf = 0;
    const int st = spasm_result(r.pr, &nf, r.placements.data(), r.traj.data(), r.cost.data(), r.success.data());
    r.n_found = nf;
    return st;
}

void scheduler_loop(spasm_server* sv) {
    cudaSetDevice(sv->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    std::vector<std::shared_ptr<Request>> active;
    spasm_batch_config cfg;
    spasm_batch_default_config(&cfg);
    for (;;) {
        std::vector<std::shared_ptr<Request>> admitted;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty() || !active.empty(); });
            if (sv->stop && sv->queue.empty() && active.empty()) break;
            while (!sv->queue.empty() && (int)(active.size() + admitted.size()) < sv->max_inflight) {
                auto& r = sv->queue.front();
                const bool alone = active.empty() && admitted.empty() && sv->in_use == 0;
                if (sv->in_use + r->bytes > sv->budget && !alone) break;   // waits for memory, in arrival order
                sv->in_use += r->bytes;
                r->state = kRunning;
                r->t_start = Clock::now();
                admitted.push_back(r);
                sv->queue.pop_front();
            }
        }
        // new requests: problem, stage 1 (device-side attempt loop), first lift
        Range epoch_range("spasm service epoch");
        for (auto& r : admitted) {
            int status = spasm_create_problem(&r->robot, &r->obs, &r->goal, &r->prm, st, &r->pr);
            if (status == SPASM_OK) status = spasm_place(r->pr);
            if (status == SPASM_OK) status = enqueue_traj_lift(r->pr, st);
            if (status != SPASM_OK) {
                const std::string msg = spasm_last_error();
                finish_request(sv, *r, status, msg);
                sv->cv_done.notify_all();
                continue;
            }
            active.push_back(r);
        }
        if (active.empty()) continue;
        // one epoch: a batched trajectory attempt of every request in flight
        std::vector<spasm_problem_t> prs;
        std::vector<int> order;
        for (size_t i = 0; i < active.size(); ++i) {
            prs.push_back(active[i]->pr);
            order.push_back((int)i);
        }
        int status = SPASM_OK;
        std::string msg;
        {
            BatchLaunch bl;
            status = prepare_batch(prs.data(), order, cfg, st, bl);
            if (status == SPASM_OK) status = enqueue_batch(bl, st);
            for (auto& r : active)
                if (status == SPASM_OK) status = enqueue_traj_epoch_end(r->pr, st);
            if (status == SPASM_OK && cudaStreamSynchronize(st) != cudaSuccess) status = SPASM_ERR_CUDA;
            if (status != SPASM_OK) msg = spasm_last_error();
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stats.epochs += 1;
            sv->stats.requests_in_epochs += (long long)active.size();
            for (auto& r : active) sv->stats.particles_in_epochs += r->prm.Q;
        }
        std::vector<std::shared_ptr<Request>> still;
        for (auto& r : active) {
            r->epochs += 1;
            if (status != SPASM_OK) {
                finish_request(sv, *r, status, msg);
                continue;
            }
            LoopCtl c{};
            if (cudaMemcpy(&c, r->pr->d_ctl, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) {
                finish_request(sv, *r, SPASM_ERR_CUDA, "reading the attempt state failed");
                continue;
            }
            bool cancel;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                cancel = r->cancel;
            }
            if (c.t_more && !cancel) {
                // another attempt: re-lift with the next attempt counter (read on the device)
                const int st2 = enqueue_traj_relift(r->pr, st);
                if (st2 == SPASM_OK) {
                    still.push_back(r);
                    continue;
                }
                finish_request(sv, *r, st2, spasm_last_error());
                continue;
            }
            if (cancel) {
                finish_request(sv, *r, SPASM_ERR_CANCELLED, "cancelled");
                continue;
            }
            // finished: FP64 check of the best P, then the outputs
            r->pr->place_pending = true;
            r->pr->traj_pending = true;
            r->pr->traj_batched = true;
            int st3 = enqueue_finish(r->pr, st);
            if (st3 == SPASM_OK) st3 = read_result(*r);
            const std::string m3 = st3 == SPASM_OK ? std::string() : std::string(spasm_last_error());
            finish_request(sv, *r, st3, m3);
        }
        active.swap(still);
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" spasm_status spasm_server_create(long long budget_bytes, int max_inflight, spasm_server_t* out) {
    if (!out || budget_bytes <= 0 || max_inflight < 1 || max_inflight > 256) return SPASM_ERR_INVALID;
    auto* sv = new spasm_server();
    cudaGetDevice(&sv->device);
    sv->budget = budget_bytes;
    sv->max_inflight = max_inflight;
    sv->scheduler = std::thread(scheduler_loop, sv);
    *out = sv;
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_submit(spasm_server_t sv, const spasm_robot* robot, const spasm_obstacles* obs,
                                            const spasm_goal* goal, const spasm_params* prm, long long* ticket) {
    if (!sv || !robot || !obs || !goal || !prm || !ticket) return SPASM_ERR_INVALID;
    if (robot->dof != 7 || goal->n_blocks < 1 || goal->n_blocks > kMaxB || prm->W < 3 || robot->n_spheres < 1 ||
        robot->n_spheres > kMaxRobotSpheres || obs->n_cuboids < 0 || obs->n_cuboids > kMaxCub || obs->n_spheres < 0 ||
        obs->n_spheres > kMaxOSph)
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
    if (spasm_problem_bytes(&r->obs, &r->goal, &r->prm, &r->bytes) != SPASM_OK) return SPASM_ERR_INVALID;
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
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                         [&] { return r->state == kDone || r->state == kCancelled; });
    return ok ? SPASM_OK : SPASM_ERR_TIMEOUT;
}

extern "C" spasm_status spasm_server_cancel(spasm_server_t sv, long long ticket) {
    if (!sv) return SPASM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return SPASM_ERR_INVALID;
    Request& r = *it->second;
    if (r.state == kQueued) {
        for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
            if ((*q)->ticket == ticket) {
                sv->queue.erase(q);
                break;
            }
        r.state = kCancelled;
        r.status = SPASM_ERR_CANCELLED;
        r.message = "cancelled";
        r.t_start = r.t_done = Clock::now();
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    } else if (r.state == kRunning) {
        r.cancel = true;   // dropped at the next epoch boundary
    }
    return SPASM_OK;
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
        if (r->state != kDone && r->state != kCancelled) return SPASM_ERR_TIMEOUT;
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
    if (it->second->state != kDone && it->second->state != kCancelled) return SPASM_ERR_INVALID;
    sv->all.erase(it);
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_get_stats(spasm_server_t sv, spasm_server_stats* out) {
    if (!sv || !out) return SPASM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->bytes_in_use = sv->in_use;
    return SPASM_OK;
}

extern "C" spasm_status spasm_server_destroy(spasm_server_t sv) {
    if (!sv) return SPASM_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->scheduler.joinable()) sv->scheduler.join();
    delete sv;
    return SPASM_OK;
}
