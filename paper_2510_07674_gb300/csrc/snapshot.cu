// Checkpoint and resume of a problem's search state.  The paper has no counterpart; a
// snapshot is what a planner keeps to answer again, or to run stage 2 again, without redoing
// stage 1.
//
// A snapshot is a header (magic, version, kind and sizes, host-side outcome, the seed, the
// size and FNV-1a digest of the payload, a digest of the obstacle set) followed by the
// payload: the device loop block (LoopCtl: the Philox key, the attempt and step counters of
// both stages, the placement and solution counts), the best P placements (P x B x 4 floats),
// and the returned solutions (P x C x 8 floats of configurations, P ranking costs, P FP64
// success flags).  Taking one completes the pending stages first; restoring one writes those
// buffers back and sets the problem's outcome, so that spasm_placements / spasm_result return
// what the snapshotted problem returned, and a spasm_optimize after a snapshot taken between
// the stages runs stage 2 from the restored placements with the restored key.
#include <cstring>
#include <string>
#include <vector>

#include "problem.h"

using namespace spasm;

namespace {

constexpr uint32_t kMagic = 0x4d535053u;   // "SPSM" little-endian
constexpr uint32_t kVersion = 1u;

struct Header {
    uint32_t magic, version;
    int32_t kind, B, C, NR, P, Q, n_cub, n_osph;
    int32_t placed, optimized, n_place, n_found, place_attempts, place_steps, traj_attempts, pad;
    uint64_t seed, payload_bytes, payload_digest, obstacle_digest;
};

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// The payload's sections in order: device pointer and bytes.
struct Section {
    void* dev;
    size_t bytes;
};

std::vector<Section> sections(spasm_problem* pr) {
    const size_t P = pr->sc.P, B = pr->sc.B, C = pr->sc.C;
    return {{pr->d_ctl, sizeof(LoopCtl)},
            {pr->d_place, P * B * 4 * sizeof(float)},
            {pr->d_rq, P * C * 8 * sizeof(float)},
            {pr->d_rcost, P * sizeof(float)},
            {pr->d_rsucc, P * sizeof(int)}};
}

size_t payload_bytes(spasm_problem* pr) {
    size_t n = 0;
    for (const Section& s : sections(pr)) n += s.bytes;
    return n;
}

uint64_t obstacle_digest(const spasm_problem* pr) {
    uint64_t h = fnv1a(pr->host_cub.data(), pr->host_cub.size() * sizeof(double));
    return fnv1a(pr->host_osph.data(), pr->host_osph.size() * sizeof(double), h);
}

Header header_of(spasm_problem* pr) {
    Header h{};
    h.magic = kMagic;
    h.version = kVersion;
    h.kind = pr->sc.kind;
    h.B = pr->sc.B; h.C = pr->sc.C; h.NR = pr->sc.NR; h.P = pr->sc.P; h.Q = pr->sc.Q;
    h.n_cub = pr->sc.n_cub; h.n_osph = pr->sc.n_osph;
    h.placed = pr->placed; h.optimized = pr->optimized;
    h.n_place = pr->n_place; h.n_found = pr->n_found;
    h.place_attempts = pr->place_attempts; h.place_steps = pr->place_steps; h.traj_attempts = pr->traj_attempts;
    h.seed = pr->sc.seed;
    h.payload_bytes = payload_bytes(pr);
    h.obstacle_digest = obstacle_digest(pr);
    return h;
}

}  // namespace

extern "C" spasm_status spasm_snapshot_bytes(spasm_problem_t pr, size_t* bytes) {
    if (!pr || !bytes) return fail(SPASM_ERR_INVALID, "null argument");
    *bytes = sizeof(Header) + payload_bytes(pr);
    return SPASM_OK;
}

extern "C" spasm_status spasm_snapshot(spasm_problem_t pr, void* host, size_t bytes) {
    if (!pr || !host) return fail(SPASM_ERR_INVALID, "null argument");
    const size_t need = sizeof(Header) + payload_bytes(pr);
    if (bytes < need) return fail(SPASM_ERR_INVALID, "snapshot buffer smaller than spasm_snapshot_bytes");
    SPASM_TRY(finalize(pr));   // the outcome of the pending stages is part of the state
    unsigned char* out = static_cast<unsigned char*>(host);
    unsigned char* pay = out + sizeof(Header);
    size_t off = 0;
    for (const Section& s : sections(pr)) {
        SPASM_CUDA(cudaMemcpyAsync(pay + off, s.dev, s.bytes, cudaMemcpyDeviceToHost, pr->stream));
        off += s.bytes;
    }
    SPASM_TRY(host_wait(pr));
    pr->stats.d2h_bytes += (long long)off;
    Header h = header_of(pr);
    h.payload_digest = fnv1a(pay, off);
    std::memcpy(out, &h, sizeof h);
    return SPASM_OK;
}

extern "C" spasm_status spasm_restore(spasm_problem_t pr, const void* host, size_t bytes) {
    if (!pr || !host) return fail(SPASM_ERR_INVALID, "null argument");
    if (bytes < sizeof(Header)) return fail(SPASM_ERR_INVALID, "snapshot shorter than its header");
    Header h;
    std::memcpy(&h, host, sizeof h);
    const Header mine = header_of(pr);
    if (h.magic != kMagic || h.version != kVersion) return fail(SPASM_ERR_INVALID, "not a snapshot of this version");
    if (h.kind != mine.kind || h.B != mine.B || h.C != mine.C || h.NR != mine.NR || h.P != mine.P || h.Q != mine.Q ||
        h.n_cub != mine.n_cub || h.n_osph != mine.n_osph || h.payload_bytes != mine.payload_bytes)
        return fail(SPASM_ERR_INVALID, "snapshot of a problem of another kind or other sizes");
    if (h.obstacle_digest != mine.obstacle_digest) return fail(SPASM_ERR_INVALID, "snapshot of another obstacle set");
    if (bytes < sizeof(Header) + h.payload_bytes) return fail(SPASM_ERR_INVALID, "snapshot shorter than its payload");
    const unsigned char* pay = static_cast<const unsigned char*>(host) + sizeof(Header);
    if (fnv1a(pay, h.payload_bytes) != h.payload_digest) return fail(SPASM_ERR_INVALID, "snapshot payload corrupted");
    LoopCtl c;
    std::memcpy(&c, pay, sizeof c);
    if (c.seed != h.seed || h.n_place < 0 || h.n_place > h.P || h.n_found < 0 || h.n_found > h.P)
        return fail(SPASM_ERR_INVALID, "snapshot header and payload disagree");
    SPASM_TRY(finalize(pr));   // nothing of this problem may still be running
    SPASM_CUDA(cudaStreamSynchronize(pr->stream));
    size_t off = 0;
    for (const Section& s : sections(pr)) {
        SPASM_CUDA(cudaMemcpyAsync(s.dev, pay + off, s.bytes, cudaMemcpyHostToDevice, pr->stream));
        off += s.bytes;
    }
    pr->sc.seed = h.seed;
    pr->prm.seed = h.seed;
    SPASM_CUDA(cudaMemcpyAsync(pr->d_sc, &pr->sc, sizeof(Scalars), cudaMemcpyHostToDevice, pr->stream));
    SPASM_TRY(host_wait(pr));   // the host buffers must outlive the copies
    pr->stats.h2d_bytes += (long long)(off + sizeof(Scalars));
    pr->placed = h.placed != 0;
    pr->optimized = h.optimized != 0;
    pr->n_place = h.n_place;
    pr->n_found = h.n_found;
    pr->place_attempts = h.place_attempts;
    pr->place_steps = h.place_steps;
    pr->traj_attempts = h.traj_attempts;
    return SPASM_OK;
}
