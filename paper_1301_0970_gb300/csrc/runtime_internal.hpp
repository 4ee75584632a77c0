// Host-side internals shared by runtime.cu (contexts, primitives) and
// register.cu (the registration pipeline: single, batched, served).
#pragma once

#include "cgdir_internal.cuh"

#include <array>
#include <atomic>
#include <cmath>
#include <map>
#include <memory>
#include <string>
#include <vector>

namespace cgdir {
namespace rt {

struct WsBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct ProfPending {
    int cls, level;
    cudaEvent_t a, b;
};

// Event pairs recorded around profiled launches, with the events they use.
struct ProfList {
    std::vector<ProfPending> recs;
    std::vector<cudaEvent_t> pool;
    void release();
};

// One instantiated CUDA graph of the device part of a registration.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    ProfList prof;
    unsigned long long launches = 0;
};

// Grow-only named device buffers; a cached graph that captured their
// addresses is dropped when one of them is reallocated.
struct WsSet {
    std::map<std::string, WsBuf> bufs;
    std::map<std::string, GraphEntry> graphs;
    unsigned long long generation = 0;
    size_t bytes() const;
};

// Kernel choices for one pyramid level shape, picked by timing (autotune.cu).
struct TunedLevel {
    int smooth_variant = 0;    // best per-step smoothing: SMOOTH_MARCH / TILE / SPLIT (0 = by size)
    int smooth_zchunk = 0;     // z chunk of the z-march smoothing (0 = default)
    int force_zchunk = 0;      // z chunk of the force stencil pass (0 = default)
    int force_width = 0;       // voxels per thread of the stencil pass: 0 = the widest, 2, 1
    float smooth_ms = 0.f, force_ms = 0.f;   // best per-step times measured
    float default_smooth_ms = 0.f, default_force_ms = 0.f;
    int fused = 0;             // the fused schedule beat the best per-step one (alone on the GPU)
    float fused_smooth_ms = 0.f, fused_force_ms = 0.f;
};
using TuneKey = std::array<int, 5>;   // nx, ny, nz, structure terms on, image storage type

struct RegPlan;   // register.cu
struct RegPlanDeleter { void operator()(RegPlan *p) const; };

// One registration's device state: its buffers, graphs, stream and the host
// copies of its result.  Slot 0 serves cgdir_register on the context stream;
// cgdir_register_batch uses one slot per case; the serving loop runs each
// admitted request in its own slot and stream.
struct Slot {
    WsSet ws;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int priority = 0;                  // of stream (served requests: by age)
    double *h_hist = nullptr;          // pinned copies of the stop state
    int *h_meta = nullptr;
    size_t h_hist_cap = 0;
    // serving
    bool busy = false;
    long long ticket = -1;
    cudaEvent_t done = nullptr;        // recorded after the request's last copy
    cudaEvent_t ready = nullptr;       // the context stream's work the request waits for
    std::unique_ptr<RegPlan, RegPlanDeleter> plan;   // of the request in flight
    float *dvf_out = nullptr;          // caller's output, copied at completion if pageable
    bool deferred_copy = false;
    const float *ufinal = nullptr;
    int status = CGDIR_OK;
};

void drop_graphs(WsSet &ws);

}  // namespace rt
}  // namespace cgdir

struct cgdir_ctx {
    unsigned prof_mask = 0;
    cgdir::rt::ProfList eager;
    std::map<std::pair<int, int>, std::pair<long long, double>> prof;
    bool use_graphs = true;
    int device = 0;
    bool plain_kernels = false;   // CGDIR_KERNELS=plain at creation: no TMA kernels
    bool fused_force = false;     // CGDIR_KERNELS=fused: one-pass TMA force kernel instead of two passes
    int smooth_variant = 0;       // SMOOTH_AUTO / MARCH / TILE (CGDIR_SMOOTH=auto|march|tile)
    bool serve_priority = true;   // served requests' streams ranked by age (CGDIR_SERVE_PRIORITY=0: off)
    int serve_schedule = 2;       // served requests' schedule (CGDIR_SERVE_SCHEDULE=shared|alone|auto:
                                  // 0|1|2): auto takes the latency one when nothing else is running
    int shared_wide_cap = 2;      // CGDIR_SHARED_WIDE_CAP=n: wide z-march CTAs per SM in batches (0: no cap)
    int force_width = 0;          // CGDIR_FORCE_WIDTH=1|2: force pass 2 voxels per thread (0: widest)
    int force_zchunk = 0;         // CGDIR_FORCE_ZCHUNK: force-pass z chunk for every level (0 = tuned / default)
    int smooth_zchunk = 0;        // CGDIR_SMOOTH_ZCHUNK: z-march smoothing z chunk (0 = tuned / default)
    long coop_max_voxels = 0;     // levels below the finest with at most this many voxels run
                                  // the cooperative level kernel (CGDIR_COOP_MAX)
    int *err_word = nullptr;      // device word set by a kernel whose bounded wait ran out
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;            // private stream the graphs are captured on
    std::vector<cudaStream_t> branch_streams;     // capture branches of a batch
    bool own_stream = false;
    size_t budget = 0;
    size_t in_use = 0;
    std::string err;
    cgdir::rt::WsSet ws;                          // scratch of the primitives
    cgdir::rt::WsSet batch;                       // graphs of cgdir_register_batch (no buffers)
    std::vector<std::unique_ptr<cgdir::rt::Slot>> slots;
    int max_slots = 8;                            // serving concurrency
    long long next_ticket = 1;
    std::map<cgdir::rt::TuneKey, cgdir::rt::TunedLevel> tuned;   // autotuned level shapes
    unsigned tune_gen = 0;                        // bumped when a choice changes (graph keys)
    bool autotune_on = false;                     // tune unseen level shapes before a registration
};

namespace cgdir {
namespace rt {

int fail(cgdir_ctx *c, int code, const std::string &msg);

#define CK(expr)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return ::cgdir::rt::fail(ctx, CGDIR_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        int r_ = (expr);               \
        if (r_ != CGDIR_OK) return r_; \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d);
    ~DeviceGuard();
};

// Event pair around one launch of class `cls` when that class is profiled.
struct ProfScope {
    ProfList *list = nullptr;
    cudaStream_t stream;
    int idx = -1;
    ProfScope(ProfList *l, unsigned mask, cudaStream_t s, int cls, int level);
    ~ProfScope();
};
void prof_collect(cgdir_ctx *ctx, const ProfList &l);

size_t round_up(size_t v, size_t a);
// Grow-only named buffer of `ws`; growing waits for `sync` (the stream that
// last used the buffer) and drops the graphs cached in `ws`.
int ws_get(cgdir_ctx *ctx, WsSet &ws, cudaStream_t sync, const char *name, size_t bytes, void **out);
inline int ws_get(cgdir_ctx *ctx, const char *name, size_t bytes, void **out) {
    return ws_get(ctx, ctx->ws, ctx->stream, name, bytes, out);
}
void ws_release(cgdir_ctx *ctx, WsSet &ws);

bool dims_ok(int nx, int ny, int nz);
bool sigma_ok(float s);
size_t elem_size(int dtype);
int *kerr(cgdir_ctx *ctx);
int check_err_word(cgdir_ctx *ctx);
int fill_force_args(cgdir_ctx *ctx, ForceArgs &a, int k, const float *lambda, const int8_t *sign,
                    float offset, int contour);
int auto_sign_impl(cgdir_ctx *ctx, const void *T0, int dtype, const uint8_t *sbits, int k, int nx, int ny,
                   int nz, int8_t *sign_host);
unsigned long long launches_now();
void launches_sub(unsigned long long n);

// Tuned (else default) kernel choices for a level shape.
// allow_fused: false for registrations that share the GPU (batches, served
// requests), which take the best per-step schedule.
SmoothChoice smooth_choice(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt, bool allow_fused);
int force_zchunk_for(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt);
bool use_level_coop(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt);
// Smallest force z chunk any tuning may choose (sizes the partial buffers).
int force_zchunk_min(int nx, int ny, int nz);
int force_width_for(const cgdir_ctx *ctx, int nx, int ny, int nz, int contour, int sdt);
// Time the candidate kernels of one level shape on synthetic data and
// record the fastest (autotune.cu).  k structures, sigma of the smoothing.
int tune_level(cgdir_ctx *ctx, int nx, int ny, int nz, int k, int contour, int sdt, float sigma);

}  // namespace rt
}  // namespace cgdir
