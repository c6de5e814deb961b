// C ABI of the SPaSM hot path (see include/spasm.h): problem set-up, the two-stage
// driver, and kernel-level entry points.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "problem.h"

using namespace spasm;

static thread_local std::string g_last_error;

namespace spasm {
cudaError_t configure_once_impl(const void* kernel, int dev, cudaError_t (*fn)(void*), void* ctx) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kernel, dev);
    if (done.count(key)) return cudaSuccess;
    const cudaError_t e = fn(ctx);
    if (e == cudaSuccess) done.insert(key);
    return e;
}
}  // namespace spasm

spasm_status spasm::fail(spasm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

// Fault injection (spasm_inject_alloc_failure): the number of allocations still to succeed
// before one fails, or -1.
static std::atomic<long long> g_alloc_countdown{-1};

// Stream-ordered allocation from the device's default memory pool: unlike cudaMalloc /
// cudaFree it does not synchronise the device, so problems created and destroyed on
// their own streams (the solver service) do not stall each other.
template <typename T>
static spasm_status dalloc(T** p, size_t count, cudaStream_t st) {
    if (count == 0) count = 1;
    if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) == 0) {
        g_alloc_countdown.store(-1);
        return fail(SPASM_ERR_NOMEM, "cudaMallocAsync: injected allocation failure");
    }
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), st);
    if (e != cudaSuccess) return fail(SPASM_ERR_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    return SPASM_OK;
}

spasm_status spasm::host_wait(spasm_problem* pr) {
    SPASM_CUDA(cudaStreamSynchronize(pr->stream));
    pr->stats.host_waits += 1;
    return SPASM_OK;
}

spasm_status spasm::check_device_error(spasm_problem* pr) {
    int err = 0;
    SPASM_CUDA(cudaMemcpyAsync(&err, pr->d_err, sizeof(int), cudaMemcpyDeviceToHost, pr->stream));
    SPASM_TRY(host_wait(pr));
    pr->stats.d2h_bytes += sizeof(int);
    if (err != 0) {
        const char* what = err == kDevTimeout ? "a bounded device wait gave up" : "a kernel rejected its sizes";
        return fail(SPASM_ERR_DEVICE, std::string("device error ") + std::to_string(err) + ": " + what);
    }
    return SPASM_OK;
}

static void free_all(spasm_problem* pr) {
    drop_graphs(pr);
    void* ptrs[] = {pr->d_cub, pr->d_osph, pr->d_err, pr->d_xs, pr->d_cost, pr->d_xm, pr->d_costm, pr->d_masked,
                    pr->d_idx, pr->d_sat, pr->d_nsat, pr->d_best, pr->d_place, pr->d_q, pr->d_lam,
                    pr->d_mu, pr->d_metrics, pr->d_tmasked, pr->d_tsat, pr->d_tnsat, pr->d_tbest, pr->d_rq,
                    pr->d_rcost, pr->d_rsucc, pr->d_cub64, pr->d_osph64, pr->d_rmet64, pr->d_tests, pr->d_sc, pr->d_chkacc,
                    pr->d_ctl};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, pr->stream);
    for (cudaEvent_t e : pr->ev)
        if (e) cudaEventDestroy(e);
    if (pr->cap) cudaStreamDestroy(pr->cap);
    if (pr->cap_body) cudaStreamDestroy(pr->cap_body);
}

// Zeroes the attempt-loop counters; a point-to-point problem has its one "placement" (the
// target) from the start.
static cudaError_t reset_loops(spasm_problem* pr) {
    LoopCtl c{};
    c.n_place = pr->sc.kind == kKindP2P ? 1 : 0;
    c.seed = pr->sc.seed;
    cudaError_t e = cudaMemcpyAsync(pr->d_ctl, &c, sizeof c, cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pr->stream);   // c lives on this stack frame
    return e;
}

extern "C" const char* spasm_last_error(void) { return g_last_error.c_str(); }

// Every device buffer of a problem with its element count, in allocation order: the one list
// that spasm_create_problem allocates and spasm_problem_bytes adds up.
template <typename F>
static void for_each_buffer(spasm_problem* pr, int B, int C, int n_cub, int n_osph, const spasm_params* prm, F&& f) {
    const size_t N = prm->N, M = prm->M, P = prm->P, Q = prm->Q, NR = 9 * (size_t)B + 3;
    f(pr->d_cub, 4 * (size_t)n_cub);
    f(pr->d_osph, (size_t)n_osph);
    f(pr->d_err, 1);
    f(pr->d_xs, 4 * (size_t)B * N);
    f(pr->d_cost, N);
    f(pr->d_idx, M);
    f(pr->d_xm, 4 * (size_t)B * M);
    f(pr->d_costm, M);
    f(pr->d_masked, M);
    f(pr->d_sat, M);
    f(pr->d_nsat, 1);
    f(pr->d_best, P);
    f(pr->d_place, P * (size_t)B * 4);
    f(pr->d_q, Q * (size_t)C * 8);
    f(pr->d_lam, Q * NR);
    f(pr->d_mu, Q);
    f(pr->d_metrics, Q * 8);
    f(pr->d_tmasked, Q);
    f(pr->d_tsat, Q);
    f(pr->d_tnsat, 1);
    f(pr->d_tbest, P);
    f(pr->d_rq, P * (size_t)C * 8);
    f(pr->d_rcost, P);
    f(pr->d_rsucc, P);
    f(pr->d_cub64, 16 * (size_t)n_cub);
    f(pr->d_osph64, 4 * (size_t)n_osph);
    f(pr->d_rmet64, 6 * P);
    f(pr->d_tests, 3);
    f(pr->d_sc, 1);
    f(pr->d_chkacc, P);
    f(pr->d_ctl, 1);
}

extern "C" spasm_status spasm_problem_bytes(const spasm_obstacles* obs, const spasm_goal* goal, const spasm_params* prm,
                                            long long* bytes) {
    if (!obs || !goal || !prm || !bytes) return fail(SPASM_ERR_INVALID, "null argument");
    const int B = goal->n_blocks;
    if (B < 1 || B > kMaxB || prm->W < 3 || obs->n_cuboids < 0 || obs->n_spheres < 0)
        return fail(SPASM_ERR_INVALID, "sizes outside the limits of spasm_create_problem");
    const int C = 2 * B * (prm->W - 1) + 1;
    spasm_problem probe;   // only its pointer members' types are used
    size_t total = 0;
    for_each_buffer(&probe, B, C, obs->n_cuboids, obs->n_spheres, prm, [&](auto*& ptr, size_t count) {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(ptr)>>;
        // the pool hands out whole allocation granules: at least one per buffer, rounded to 512 bytes
        total += ((std::max<size_t>(count, 1) * sizeof(T) + 511) / 512) * 512;
    });
    *bytes = (long long)total;
    return SPASM_OK;
}

// The joint layout the analytic lift IK solves (the Franka arm's): twists (0, -pi/2, pi/2,
// pi/2, -pi/2, pi/2, pi/2), a_0 = a_1 = a_2 = a_5 = 0, d_1 = d_3 = d_5 = d_6 = 0, and an
// elbow whose two links are not both of zero length.
static bool franka_layout(const double* dh) {
    const double h = 1.5707963267948966;
    const double alpha[7] = {0.0, -h, h, h, -h, h, h};
    for (int k = 0; k < 7; ++k)
        if (std::fabs(dh[4 * k + 1] - alpha[k]) > 1e-9) return false;
    for (int k : {0, 1, 2, 5})
        if (dh[4 * k] != 0.0) return false;
    for (int k : {1, 3, 5, 6})
        if (dh[4 * k + 2] != 0.0) return false;
    const double a3 = dh[12], a4 = dh[16], d2 = dh[10], d4 = dh[18];
    return std::hypot(a3 * a4 + d2 * d4, d2 * a4 - a3 * d4) > 0.0;
}

static spasm_status create_problem_impl(const spasm_robot* robot, const spasm_obstacles* obs, const spasm_goal* goal,
                                        const spasm_params* prm, void* cuda_stream, spasm_problem_t* out) {
    Range range("spasm create problem");
    if (!robot || !obs || !goal || !prm || !out) return fail(SPASM_ERR_INVALID, "null argument");
    *out = nullptr;
    if (robot->dof != 7) return fail(SPASM_ERR_INVALID, "dof must be 7");
    if (robot->n_spheres < 1 || robot->n_spheres > kMaxRobotSpheres)
        return fail(SPASM_ERR_INVALID, "robot sphere count outside 1..56");
    if (obs->n_cuboids < 0 || obs->n_cuboids > kMaxCub) return fail(SPASM_ERR_INVALID, "cuboid count outside 0..256");
    if (obs->n_spheres < 0 || obs->n_spheres > kMaxOSph) return fail(SPASM_ERR_INVALID, "obstacle sphere count outside 0..64");
    const int B = goal->n_blocks;
    if (B < 1 || B > kMaxB) return fail(SPASM_ERR_INVALID, "n_blocks outside 1..16");
    if (prm->W < 3) return fail(SPASM_ERR_INVALID, "W must be >= 3");
    const int S = prm->W - 1, C = 2 * B * S + 1;
    if (C > kMaxC) return fail(SPASM_ERR_INVALID, "too many configurations (2B(W-1)+1 > 1024)");
    if (prm->N < 1 || prm->N > 32768 || prm->M < 1 || prm->M > 8192 || prm->M > prm->N)
        return fail(SPASM_ERR_INVALID, "need 1 <= M <= N, N <= 32768, M <= 8192");
    if (prm->P < 1 || prm->P > prm->M || prm->Q < 1 || prm->Q > 1 << 20)
        return fail(SPASM_ERR_INVALID, "need 1 <= P <= M and 1 <= Q");
    if (prm->K_lin < 1 || prm->K_quad < 0 || prm->K_traj < 1 || prm->K_ik < 0)
        return fail(SPASM_ERR_INVALID, "step counts must be positive");
    if (prm->ik_mode != 0 && prm->ik_mode != 1) return fail(SPASM_ERR_INVALID, "ik_mode must be 0 or 1");
    if (prm->ik_mode == 1 && !franka_layout(robot->dh))
        return fail(SPASM_ERR_INVALID, "ik_mode 1 needs the Franka joint layout (alpha, zero a and d entries)");
    for (int i = 0; i < robot->n_spheres; ++i)
        if (robot->sphere_link[i] < 0 || robot->sphere_link[i] > 7) return fail(SPASM_ERR_INVALID, "sphere_link outside 0..7");

    spasm_problem* pr = new spasm_problem();
    pr->prm = *prm;
    pr->stream = static_cast<cudaStream_t>(cuda_stream);
    Scalars& sc = pr->sc;
    std::memset(&sc, 0, sizeof sc);
    sc.B = B; sc.S = S; sc.C = C; sc.NR = 9 * B + 3;
    sc.n_rsph = robot->n_spheres; sc.n_cub = obs->n_cuboids; sc.n_osph = obs->n_spheres;
    sc.K_lin = prm->K_lin; sc.K_quad = prm->K_quad; sc.K_traj = prm->K_traj; sc.K_al = prm->K_al; sc.K_ik = prm->K_ik;
    sc.N = prm->N; sc.M = prm->M; sc.P = prm->P; sc.Q = prm->Q;
    for (int k = 0; k < 7; ++k) {
        const double* row = robot->dh + 4 * k;
        sc.a[k] = (float)row[0];
        sc.ca[k] = (float)std::cos(row[1]);
        sc.sa[k] = (float)std::sin(row[1]);
        sc.d[k] = (float)row[2];
        sc.th0[k] = (float)row[3];
        sc.qlo[k] = (float)robot->qlim[2 * k];
        sc.qhi[k] = (float)robot->qlim[2 * k + 1];
        sc.q_home[k] = (float)robot->q_home[k];
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) sc.ee_R[3 * i + j] = (float)robot->ee[4 * i + j];
        sc.ee_p[i] = (float)robot->ee[4 * i + 3];
    }
    for (int i = 0; i < robot->n_spheres; ++i) {
        const double* s = robot->sphere + 4 * i;
        sc.rsph[i] = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[3]);
        sc.rlink[i] = robot->sphere_link[i];
    }
    for (int l = 0; l < 8; ++l) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        bool any = false;
        for (int i = 0; i < robot->n_spheres; ++i) {
            if (robot->sphere_link[i] != l) continue;
            const double* s = robot->sphere + 4 * i;
            for (int k = 0; k < 3; ++k) { lo[k] = std::fmin(lo[k], s[k] - s[3]); hi[k] = std::fmax(hi[k], s[k] + s[3]); }
            any = true;
        }
        // the pad keeps the box conservative under the FP32 rounding of its world transform
        const double pad = 1e-5;
        sc.lbox_c[l] = any ? make_float4((float)(0.5 * (lo[0] + hi[0])), (float)(0.5 * (lo[1] + hi[1])),
                                         (float)(0.5 * (lo[2] + hi[2])), 0.f)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        sc.lbox_h[l] = any ? make_float4((float)(0.5 * (hi[0] - lo[0]) + pad), (float)(0.5 * (hi[1] - lo[1]) + pad),
                                         (float)(0.5 * (hi[2] - lo[2]) + pad), 0.f)
                           : make_float4(-1.f, -1.f, -1.f, 0.f);
    }
    {
        // Joint j turns about the axis through the origin of frame j+1; a point of link l > j lies
        // within sum_{k=j+1}^{l-1} |t_k| + |p| of that origin (t_k: origin of frame k+1 in frame
        // k, |t_k| = hypot(a_k, d_k); p: the point in frame l), and a held-block sphere centre
        // within |ee_p| + h_z + grasp_off + |h|/2 of frame 7's origin.  Moving one joint at a time,
        // a point travels at most |dq_j| times its distance from axis j.
        double reach[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool has[8] = {false, false, false, false, false, false, false, false};
        for (int i = 0; i < robot->n_spheres; ++i) {
            const double* v = robot->sphere + 4 * i;
            const int l = robot->sphere_link[i];
            reach[l] = std::fmax(reach[l], std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
            has[l] = true;
        }
        const double* E = robot->ee;
        double held = 0.0;
        for (int i = 0; i < B; ++i) {
            const double* h = goal->half_ext + 3 * i;
            held = std::fmax(held, h[2] + goal->grasp_off + 0.5 * std::sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]));
        }
        reach[7] = std::fmax(reach[7], std::sqrt(E[3] * E[3] + E[7] * E[7] + E[11] * E[11]) + held);
        has[7] = true;
        for (int j = 0; j < 7; ++j) {
            double L = 0.0, path = 0.0;
            for (int l = j + 1; l <= 7; ++l) {
                if (l > j + 1) path += std::hypot(robot->dh[4 * (l - 1)], robot->dh[4 * (l - 1) + 2]);
                if (has[l]) L = std::fmax(L, path + reach[l]);
            }
            sc.sweep[j] = (float)(L * (1.0 + 1e-5) + 1e-5);
        }
    }
    double z = goal->z_table;
    for (int i = 0; i < B; ++i) {
        const double* h = goal->half_ext + 3 * i;
        const double* p = goal->init_pose + 4 * i;
        double hm = std::fmin(h[0], std::fmin(h[1], h[2]));
        sc.half[i] = make_float4((float)h[0], (float)h[1], (float)h[2], (float)(0.5 * hm));
        sc.init[i] = make_float4((float)p[0], (float)p[1], (float)p[2], (float)p[3]);
        sc.zt[i] = (float)(z + h[2]);
        z += 2.0 * h[2];
        sc.zlo[i] = (float)std::fmax(goal->goal_box[2], goal->z_table + h[2]);
    }
    for (int k = 0; k < 3; ++k) { sc.box_lo[k] = (float)goal->goal_box[k]; sc.box_hi[k] = (float)goal->goal_box[3 + k]; }
    sc.z_table = (float)goal->z_table;
    sc.grasp_off = (float)goal->grasp_off;
    sc.eta_init = (float)prm->eta_init; sc.alpha = (float)prm->alpha; sc.eta_traj = (float)prm->eta_traj;
    sc.eps = (float)prm->eps; sc.eps_start = (float)prm->eps_start;
    sc.w_stable = (float)prm->w_stable; sc.w_height = (float)prm->w_height; sc.w_coll = (float)prm->w_coll;
    sc.w_start = (float)prm->w_start; sc.w_arm = (float)prm->w_arm; sc.w_block = (float)prm->w_block;
    sc.w_path = (float)prm->w_path; sc.w_jl = (float)prm->w_jl;
    {
        const float w6[6] = {sc.w_start, sc.w_height, sc.w_stable, sc.w_coll, sc.w_arm, sc.w_block};
        for (int k = 0; k < 6; ++k) sc.sqw[k] = std::sqrt(w6[k]);   // IEEE float sqrt, as sqrtf on the device
    }
    sc.mu0 = (float)prm->mu0; sc.mu_max = (float)prm->mu_max; sc.ik_damp = (float)prm->ik_damp;
    sc.ik_mode = prm->ik_mode;
    sc.seed = prm->seed;

    // environment tables: cuboid = centre (+ bounding radius), then columns of R with half extents
    std::vector<float4> cub(4 * (size_t)sc.n_cub);
    for (int o = 0; o < sc.n_cub; ++o) {
        const double* c = obs->cuboid + 15 * o;
        const double *R = c + 3, *h = c + 12;
        const double rad = std::sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
        cub[4 * o] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)rad);
        for (int k = 0; k < 3; ++k) cub[4 * o + 1 + k] = make_float4((float)R[k], (float)R[3 + k], (float)R[6 + k], (float)h[k]);
    }
    std::vector<float4> osph((size_t)sc.n_osph);
    for (int o = 0; o < sc.n_osph; ++o) {
        const double* s = obs->sphere + 4 * o;
        osph[o] = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[3]);
    }
    pr->host_cub.assign(obs->cuboid, obs->cuboid + 15 * (size_t)sc.n_cub);
    std::vector<double> cub64(16 * (size_t)sc.n_cub), osph64(4 * (size_t)sc.n_osph);
    for (int o = 0; o < sc.n_cub; ++o) {
        const double* c = obs->cuboid + 15 * o;
        double* d = &cub64[16 * (size_t)o];
        d[0] = c[0]; d[1] = c[1]; d[2] = c[2]; d[3] = 0.0;
        for (int k = 0; k < 3; ++k) {
            d[4 + 4 * k] = c[3 + k]; d[5 + 4 * k] = c[6 + k]; d[6 + 4 * k] = c[9 + k]; d[7 + 4 * k] = c[12 + k];
        }
    }
    for (int o = 0; o < 4 * sc.n_osph; ++o) osph64[o] = obs->sphere[o];
    {
        Scalars64& q = pr->s64;
        std::memset(&q, 0, sizeof q);
        q.B = B; q.S = S; q.C = C; q.n_rsph = sc.n_rsph; q.n_cub = sc.n_cub; q.n_osph = sc.n_osph;
        for (int k = 0; k < 7; ++k) {
            const double* row = robot->dh + 4 * k;
            q.a[k] = row[0]; q.ca[k] = std::cos(row[1]); q.sa[k] = std::sin(row[1]); q.d[k] = row[2]; q.th0[k] = row[3];
            // the limits as the FP32 path holds them: a joint clamped to its limit in FP32 sits at
            // the float nearest the limit, which may lie a rounding step beyond the double value
            q.qlo[k] = (double)(float)robot->qlim[2 * k]; q.qhi[k] = (double)(float)robot->qlim[2 * k + 1];
        }
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) q.ee_R[3 * i + j] = robot->ee[4 * i + j];
            q.ee_p[i] = robot->ee[4 * i + 3];
        }
        for (int i = 0; i < sc.n_rsph; ++i) {
            for (int k = 0; k < 4; ++k) q.rsph[i][k] = robot->sphere[4 * i + k];
            q.rlink[i] = robot->sphere_link[i];
        }
        double zz = goal->z_table;
        for (int i = 0; i < B; ++i) {
            const double* hh = goal->half_ext + 3 * i;
            for (int k = 0; k < 3; ++k) q.half[i][k] = hh[k];
            q.hmin[i] = std::fmin(hh[0], std::fmin(hh[1], hh[2]));
            for (int k = 0; k < 4; ++k) q.init[i][k] = goal->init_pose[4 * i + k];
            q.zt[i] = zz + hh[2];
            zz += 2.0 * hh[2];
        }
        q.grasp_off = goal->grasp_off; q.eps = prm->eps; q.eps_start = prm->eps_start;
    }
    pr->host_osph.assign(obs->sphere, obs->sphere + 4 * (size_t)sc.n_osph);

    spasm_status st = SPASM_OK;
    for_each_buffer(pr, B, C, sc.n_cub, sc.n_osph, prm, [&](auto*& ptr, size_t count) {
        if (st == SPASM_OK) st = dalloc(&ptr, count, pr->stream);
    });
    for (auto& ev : pr->ev)
        if (st == SPASM_OK && cudaEventCreate(&ev) != cudaSuccess) st = fail(SPASM_ERR_CUDA, "cudaEventCreate failed");
    // streams the attempt-loop graphs are captured on (the problem's own stream may be the
    // legacy default stream, which cannot be captured)
    if (st == SPASM_OK && (cudaStreamCreateWithFlags(&pr->cap, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaStreamCreateWithFlags(&pr->cap_body, cudaStreamNonBlocking) != cudaSuccess))
        st = fail(SPASM_ERR_CUDA, "cudaStreamCreateWithFlags failed");
    if (st != SPASM_OK) { free_all(pr); delete pr; return st; }
    pr->tab.cub = pr->d_cub;
    pr->tab.osph = pr->d_osph;
    cudaError_t e = cudaSuccess;
    if (!cub.empty()) e = cudaMemcpyAsync(pr->d_cub, cub.data(), cub.size() * sizeof(float4), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess && !osph.empty())
        e = cudaMemcpyAsync(pr->d_osph, osph.data(), osph.size() * sizeof(float4), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess && !cub64.empty())
        e = cudaMemcpyAsync(pr->d_cub64, cub64.data(), cub64.size() * sizeof(double), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess && !osph64.empty())
        e = cudaMemcpyAsync(pr->d_osph64, osph64.data(), osph64.size() * sizeof(double), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr->d_sc, &pr->sc, sizeof(Scalars), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr->d_err, 0, sizeof(int), pr->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr->d_chkacc, 0, sizeof(CheckAcc) * (size_t)prm->P, pr->stream);
    if (e == cudaSuccess) e = reset_loops(pr);
    if (e != cudaSuccess) {
        free_all(pr);
        delete pr;
        return fail(SPASM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    pr->stats.h2d_bytes += (long long)(cub.size() * sizeof(float4) + osph.size() * sizeof(float4) +
                                       cub64.size() * sizeof(double) + osph64.size() * sizeof(double));
    const size_t need = traj_smem_bytes(sc);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (max_smem > 0 && need > (size_t)max_smem) {
        free_all(pr);
        delete pr;
        return fail(SPASM_ERR_INVALID, "problem too large for the per-CTA shared memory of the trajectory kernel");
    }
    *out = pr;
    return SPASM_OK;
}

// Builds the stage graphs of a new problem (a failure destroys it).
static spasm_status finish_create(spasm_problem_t pr, spasm_problem_t* out) {
    const spasm_status st = prepare_graphs(pr);
    if (st != SPASM_OK) {
        const std::string msg = spasm_last_error();
        spasm_destroy_problem(pr);
        return fail(st, msg);
    }
    *out = pr;
    return SPASM_OK;
}

extern "C" spasm_status spasm_create_problem(const spasm_robot* robot, const spasm_obstacles* obs,
                                             const spasm_goal* goal, const spasm_params* prm, void* cuda_stream,
                                             spasm_problem_t* out) {
    if (!out) return fail(SPASM_ERR_INVALID, "null argument");
    spasm_problem_t pr = nullptr;
    SPASM_TRY(create_problem_impl(robot, obs, goal, prm, cuda_stream, &pr));
    return finish_create(pr, out);
}

extern "C" spasm_status spasm_create_packing(const spasm_robot* robot, const spasm_packing* pk,
                                             const spasm_params* prm, void* cuda_stream, spasm_problem_t* out) {
    if (!pk || !out) return fail(SPASM_ERR_INVALID, "null argument");
    *out = nullptr;
    const int B = pk->n_blocks;
    if (B < 1 || B > kMaxB || !pk->n_cells || !pk->cell || !pk->region)
        return fail(SPASM_ERR_INVALID, "packing: n_blocks outside 1..16 or a null table");
    int total = 0;
    for (int i = 0; i < B; ++i) {
        if (pk->n_cells[i] < 1 || pk->n_cells[i] > 8) return fail(SPASM_ERR_INVALID, "packing: 1..8 cells per block");
        total += pk->n_cells[i];
    }
    if (total > kMaxCells) return fail(SPASM_ERR_INVALID, "packing: more than 64 cells");
    const double u = pk->cell_size, zs = pk->z_star;
    const double* rg = pk->region;
    if (!(u > 0.0) || !(pk->z_span >= 0.0) || !(rg[2] > rg[0]) || !(rg[3] > rg[1]))
        return fail(SPASM_ERR_INVALID, "packing: bad cell size, height range or region");
    // the walls: slabs of thickness u and height u just outside the region
    const double xc = 0.5 * (rg[0] + rg[2]), yc = 0.5 * (rg[1] + rg[3]);
    const double hx = 0.5 * (rg[2] - rg[0]) + u, hy = 0.5 * (rg[3] - rg[1]) + u;
    const double wc[4][3] = {{rg[0] - 0.5 * u, yc, zs}, {rg[2] + 0.5 * u, yc, zs}, {xc, rg[1] - 0.5 * u, zs},
                             {xc, rg[3] + 0.5 * u, zs}};
    const double wh[4][3] = {{0.5 * u, hy, 0.5 * u}, {0.5 * u, hy, 0.5 * u}, {hx, 0.5 * u, 0.5 * u}, {hx, 0.5 * u, 0.5 * u}};
    std::vector<double> walls(4 * 15, 0.0);
    for (int w = 0; w < 4; ++w) {
        double* r = walls.data() + 15 * w;
        for (int k = 0; k < 3; ++k) { r[k] = wc[w][k]; r[12 + k] = wh[w][k]; }
        r[3] = r[7] = r[11] = 1.0;
    }
    std::vector<double> half(3 * B, 0.5 * u), init(4 * B, 0.0);
    const double box[6] = {rg[0], rg[1], zs, rg[2], rg[3], zs + pk->z_span};
    spasm_obstacles obs{4, walls.data(), 0, nullptr};
    spasm_goal goal{B, half.data(), init.data(), box, zs - 0.5 * u, 0.0};
    spasm_problem_t pr = nullptr;
    SPASM_TRY(create_problem_impl(robot, &obs, &goal, prm, cuda_stream, &pr));
    Scalars& sc = pr->sc;
    sc.kind = kKindPack;
    sc.n_cells = total;
    sc.cell_size = (float)u;
    sc.z_star = (float)zs;
    int k = 0;
    for (int i = 0; i < B; ++i) {
        sc.cell_start[i] = k;
        double reach = 0.0;
        for (int c = 0; c < pk->n_cells[i]; ++c, ++k) {
            const double ox = pk->cell[2 * k], oy = pk->cell[2 * k + 1];
            sc.cell[k] = make_float2((float)ox, (float)oy);
            sc.cell_block[k] = (signed char)i;
            reach = std::fmax(reach, std::sqrt(ox * ox + oy * oy));
        }
        // farthest point of the block's cubes from its origin (padded against rounding)
        sc.cell_reach[i] = (float)(reach + 0.5 * std::sqrt(3.0) * u + 1e-5);
    }
    sc.cell_start[B] = k;
    cudaError_t e = cudaMemcpyAsync(pr->d_sc, &pr->sc, sizeof(Scalars), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pr->stream);
    if (e != cudaSuccess) {
        spasm_destroy_problem(pr);
        return fail(SPASM_ERR_CUDA, std::string("create_packing: ") + cudaGetErrorString(e));
    }
    return finish_create(pr, out);
}

extern "C" spasm_status spasm_create_p2p(const spasm_robot* robot, const spasm_obstacles* obs, const double* target,
                                         const spasm_params* prm, void* cuda_stream, spasm_problem_t* out) {
    if (!target || !out || !prm) return fail(SPASM_ERR_INVALID, "null argument");
    *out = nullptr;
    const double half[3] = {0.0, 0.0, 0.0};
    const double box[6] = {target[0] - 0.1, target[1] - 0.1, target[2], target[0] + 0.1, target[1] + 0.1, target[2] + 0.1};
    spasm_goal goal{1, half, target, box, target[2], 0.0};
    spasm_problem_t pr = nullptr;
    SPASM_TRY(create_problem_impl(robot, obs, &goal, prm, cuda_stream, &pr));
    // one transit segment: C = W configurations; stage 1 does not apply
    pr->sc.kind = kKindP2P;
    pr->sc.C = pr->sc.S + 1;
    pr->s64.C = pr->sc.C;
    pr->s64.p2p = 1;
    pr->placed = true;
    pr->n_place = 1;
    cudaError_t e = cudaMemsetAsync(pr->d_place, 0, sizeof(float) * 4, pr->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr->d_sc, &pr->sc, sizeof(Scalars), cudaMemcpyHostToDevice, pr->stream);
    if (e == cudaSuccess) e = reset_loops(pr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pr->stream);
    if (e != cudaSuccess) {
        spasm_destroy_problem(pr);
        return fail(SPASM_ERR_CUDA, std::string("create_p2p: ") + cudaGetErrorString(e));
    }
    return finish_create(pr, out);
}

extern "C" spasm_status spasm_placements(spasm_problem_t pr, int* n_place, double* placements) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    SPASM_TRY(finalize(pr));
    std::vector<float> tmp(placements ? (size_t)pr->sc.P * pr->sc.B * 4 : 0);
    if (placements)
        SPASM_CUDA(cudaMemcpyAsync(tmp.data(), pr->d_place, tmp.size() * sizeof(float), cudaMemcpyDeviceToHost, pr->stream));
    SPASM_TRY(host_wait(pr));
    pr->stats.d2h_bytes += (long long)(tmp.size() * sizeof(float));
    if (n_place) *n_place = pr->placed ? pr->n_place : 0;
    for (size_t i = 0; i < tmp.size(); ++i) placements[i] = tmp[i];
    if (!pr->placed || pr->n_place == 0) return fail(SPASM_ERR_NOSOLUTION, "no placements");
    return SPASM_OK;
}

extern "C" spasm_status spasm_destroy_problem(spasm_problem_t pr) {
    if (!pr) return SPASM_OK;
    cudaStreamSynchronize(pr->stream);
    free_all(pr);
    delete pr;
    return SPASM_OK;
}

extern "C" spasm_status spasm_sizes(spasm_problem_t pr, int* C, int* NR) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    if (C) *C = pr->sc.C;
    if (NR) *NR = pr->sc.NR;
    return SPASM_OK;
}

extern "C" spasm_status spasm_result(spasm_problem_t pr, int* n_found, double* placements, double* traj, double* cost,
                                     int* success) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    const Scalars& sc = pr->sc;
    const int P = sc.P, B = sc.B, C = sc.C;
    SPASM_TRY(finalize(pr));
    std::vector<float> tp(placements ? (size_t)P * B * 4 : 0), tq(traj ? (size_t)P * C * 8 : 0), tc(cost ? P : 0);
    if (placements)
        SPASM_CUDA(cudaMemcpyAsync(tp.data(), pr->d_place, tp.size() * sizeof(float), cudaMemcpyDeviceToHost, pr->stream));
    if (traj) SPASM_CUDA(cudaMemcpyAsync(tq.data(), pr->d_rq, tq.size() * sizeof(float), cudaMemcpyDeviceToHost, pr->stream));
    if (cost) SPASM_CUDA(cudaMemcpyAsync(tc.data(), pr->d_rcost, tc.size() * sizeof(float), cudaMemcpyDeviceToHost, pr->stream));
    if (success) SPASM_CUDA(cudaMemcpyAsync(success, pr->d_rsucc, P * sizeof(int), cudaMemcpyDeviceToHost, pr->stream));
    SPASM_TRY(host_wait(pr));
    pr->stats.d2h_bytes += (long long)((tp.size() + tq.size() + tc.size()) * sizeof(float) + (success ? P * sizeof(int) : 0));
    if (n_found) *n_found = pr->optimized ? pr->n_found : 0;
    for (size_t i = 0; i < tp.size(); ++i) placements[i] = tp[i];
    if (traj)
        for (int r = 0; r < P; ++r)
            for (int t = 0; t < C; ++t)
                for (int j = 0; j < 7; ++j) traj[((size_t)r * C + t) * 7 + j] = tq[((size_t)r * C + t) * 8 + j];
    for (size_t r = 0; r < tc.size(); ++r) cost[r] = tc[r];
    if (!pr->optimized || pr->n_found == 0) return fail(SPASM_ERR_NOSOLUTION, "no solution");
    return SPASM_OK;
}

// ---------------------------------------------------------------------------------- kernel level
extern "C" spasm_status spasm_place_sample(spasm_problem_t pr, int n, uint32_t attempt, float* x, float* cost) {
    if (!pr || n < 0 || (n > 0 && (!x || !cost))) return fail(SPASM_ERR_INVALID, "bad arguments");
    SPASM_CUDA(launch_place_sample_cost(pr->sc, pr->tab, n, attempt, x, cost, pr->d_err, pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_place_eval(spasm_problem_t pr, int n, const float* x, int quadratic, float* cost,
                                         float* grad, float* metrics, float* terms) {
    if (!pr || n < 0 || (n > 0 && !x)) return fail(SPASM_ERR_INVALID, "bad arguments");
    SPASM_CUDA(launch_place_eval(pr->sc, pr->tab, n, x, quadratic, cost, grad, metrics, terms, pr->d_err, pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_place_descend(spasm_problem_t pr, int n, float* x, int k_lin, int k_quad, float* cost,
                                            int* sat) {
    if (!pr || n < 0 || (n > 0 && !x) || k_lin < 1 || k_quad < 0) return fail(SPASM_ERR_INVALID, "bad arguments");
    if (n == 0) return SPASM_OK;
    // each warp reads its own particle's column before writing it back: in place is safe
    SPASM_CUDA(launch_place_descend(pr->sc, pr->tab, n, x, n, nullptr, x, k_lin, k_quad, cost, sat, nullptr, pr->d_err,
                                    pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_select_topk(spasm_problem_t pr, int n, const float* cost, int k, int* idx) {
    if (!pr || n < 0 || k < 0 || n > 32768 || k > 8192 || (n > 0 && (!cost || !idx)))
        return fail(SPASM_ERR_INVALID, "bad arguments (n <= 32768, k <= 8192)");
    SPASM_CUDA(launch_topk(cost, n, k, idx, nullptr, pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_lift(spasm_problem_t pr, int n, const float* placements, int n_place, uint32_t attempt,
                                   float* q) {
    if (!pr || n < 0 || n_place < 1 || (n > 0 && (!placements || !q))) return fail(SPASM_ERR_INVALID, "bad arguments");
    SPASM_CUDA(launch_lift(pr->sc, n, placements, n_place, attempt, q, pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_traj_eval(spasm_problem_t pr, int n, const float* q, const float* lam, const float* mu,
                                        float* L, float* grad, float* groups, float* h) {
    if (!pr || n < 0 || (n > 0 && !q)) return fail(SPASM_ERR_INVALID, "bad arguments");
    TrajIO io{};
    io.q = const_cast<float*>(q);
    io.lam = const_cast<float*>(lam);
    io.mu = const_cast<float*>(mu);
    io.L = L; io.grad = grad; io.groups = groups; io.h = h;
    SPASM_CUDA(launch_traj(pr->sc, pr->tab, n, kTrajModeEval, io, pr->d_err, pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_traj_descend(spasm_problem_t pr, int n, float* q, float* lam, float* mu, int k_steps,
                                           int init_multipliers, float* metrics, int* sat) {
    if (!pr || n < 0 || k_steps < 1 || (n > 0 && !q)) return fail(SPASM_ERR_INVALID, "bad arguments");
    if (!init_multipliers && (!lam || !mu)) return fail(SPASM_ERR_INVALID, "lam and mu required");
    TrajIO io{};
    io.q = q; io.lam = lam; io.mu = mu; io.metrics = metrics; io.sat = sat;
    io.k_steps = k_steps; io.init_multipliers = init_multipliers;
    SPASM_CUDA(launch_traj(pr->sc, pr->tab, n, kTrajModeDescend, io, pr->d_err, pr->stream));
    return SPASM_OK;
}

extern "C" spasm_status spasm_traj_check(spasm_problem_t pr, int n, const float* q, double* metrics, int* ok) {
    if (!pr || n < 0 || (n > 0 && (!q || !metrics || !ok))) return fail(SPASM_ERR_INVALID, "bad arguments");
    // the accumulators of the split check hold P rows: check in chunks of at most P
    const int P = pr->sc.P, C = pr->sc.C;
    for (int off = 0; off < n; off += P) {
        const int k = n - off < P ? n - off : P;
        SPASM_CUDA(launch_check64(pr->s64, pr->d_cub64, pr->d_osph64, q + (size_t)off * C * 8, nullptr, k,
                                  metrics + (size_t)off * 6, ok + off, pr->d_chkacc, pr->stream));
    }
    return SPASM_OK;
}

extern "C" spasm_status spasm_set_kernel_config(spasm_problem_t pr, const spasm_kernel_config* cfg) {
    if (!pr || !cfg) return fail(SPASM_ERR_INVALID, "null argument");
    if (cfg->sphere_tiling < 0 || cfg->sphere_tiling > 1 || cfg->particles_per_cta < 1 || cfg->particles_per_cta > 2)
        return fail(SPASM_ERR_INVALID, "sphere_tiling must be 0 or 1 and particles_per_cta 1 or 2");
    int dev = 0, max_smem = 0;
    SPASM_CUDA(cudaGetDevice(&dev));
    SPASM_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (traj_cta_smem_bytes(pr->sc, cfg->particles_per_cta) > (size_t)max_smem)
        return fail(SPASM_ERR_INVALID, "the shared memory of that many particles per CTA does not fit this problem");
    SPASM_TRY(finalize(pr));
    SPASM_TRY(host_wait(pr));
    pr->sc.sphere_tiling = cfg->sphere_tiling;
    pr->sc.particles_per_cta = cfg->particles_per_cta;
    SPASM_CUDA(cudaMemcpyAsync(pr->d_sc, &pr->sc, sizeof(Scalars), cudaMemcpyHostToDevice, pr->stream));
    SPASM_TRY(host_wait(pr));
    drop_graphs(pr);   // their launches hold the old shape
    return prepare_graphs(pr);
}

extern "C" spasm_status spasm_traj_residency(spasm_problem_t pr, int* single, int* batched) {
    if (!pr || !single || !batched) return fail(SPASM_ERR_INVALID, "null argument");
    *single = traj_ctas_per_sm(pr->sc);
    *batched = traj_batch_ctas_per_sm(traj_smem_bytes(pr->sc), pr->sc.sphere_tiling,
                                      pr->sc.particles_per_cta == 2 ? 2 : 1);
    return SPASM_OK;
}

extern "C" spasm_status spasm_synchronize(spasm_problem_t pr) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    SPASM_TRY(finalize(pr));
    return check_device_error(pr);
}

extern "C" spasm_status spasm_inject_alloc_failure(int nth) {
    if (nth < -1) return fail(SPASM_ERR_INVALID, "nth must be >= -1");
    g_alloc_countdown.store(nth);
    return SPASM_OK;
}

extern "C" spasm_status spasm_set_seed(spasm_problem_t pr, uint64_t seed) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    SPASM_TRY(finalize(pr));
    SPASM_CUDA(cudaStreamSynchronize(pr->stream));
    pr->sc.seed = seed;
    pr->prm.seed = seed;
    // the stage graphs read the key from the loop block on the device, so they stay valid
    SPASM_CUDA(cudaMemcpyAsync(pr->d_sc, &pr->sc, sizeof(Scalars), cudaMemcpyHostToDevice, pr->stream));
    SPASM_CUDA(reset_loops(pr));
    pr->optimized = false;
    pr->placed = pr->sc.kind == kKindP2P;   // a point-to-point problem has no stage 1
    pr->n_place = pr->placed ? 1 : 0;
    pr->n_found = 0;
    return SPASM_OK;
}

extern "C" spasm_status spasm_set_timing(spasm_problem_t pr, int enable) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    pr->timing = enable != 0;
    return SPASM_OK;
}

extern "C" spasm_status spasm_get_stats(spasm_problem_t pr, spasm_stats* out) {
    if (!pr || !out) return fail(SPASM_ERR_INVALID, "null argument");
    SPASM_TRY(finalize(pr));
    *out = pr->stats;
    return SPASM_OK;
}

extern "C" spasm_status spasm_reset_stats(spasm_problem_t pr) {
    if (!pr) return fail(SPASM_ERR_INVALID, "null problem");
    pr->stats = spasm_stats{};
    return SPASM_OK;
}

// accessors used by the static-scratch entry point (noalloc.cu)
namespace spasm {
const Scalars& problem_scalars(const spasm_problem* pr) { return pr->sc; }
DevTables problem_tables(const spasm_problem* pr) { return pr->tab; }
cudaStream_t problem_stream(const spasm_problem* pr) { return pr->stream; }
int* problem_error_word(spasm_problem* pr) { return pr->d_err; }
spasm_status set_last_error(spasm_status st, const std::string& msg) { return fail(st, msg); }
}  // namespace spasm
