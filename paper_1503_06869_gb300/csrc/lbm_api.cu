// lbm_api.cu -- the C interface declared in include/lbm.h: contexts, device
// memory, the order of the kernels in a time step (Sec. 4.3: sweep with
// bounce-back and momentum exchange, rigid-body update, re-mapping), CUDA
// graph replay, sweep timing and the launch-shape autotuner.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbm;

// Extra elements per population plane (a multiple of 64 keeps every plane
// start on a 256-byte boundary in all storage forms).
#ifndef LBM_PLANE_PAD
#define LBM_PLANE_PAD 0
#endif

struct lbm_ctx {
    lbm_precision prec = LBM_F32;
    int device = 0;                 // CUDA device current at creation; every call runs with it current
    int esize = 4;
    cudaStream_t stream = nullptr;
    void *(*dev_alloc)(size_t, void *) = nullptr;
    void (*dev_free)(void *, void *) = nullptr;
    void *user = nullptr;
    std::vector<void *> owned;      // every device allocation of the context
    size_t device_bytes = 0;

    int nlat = 0;
    std::vector<LatDev> lat_h;
    LatDev *lat_d = nullptr;
    long long ncells = 0, f_elems = 0;
    void *f = nullptr;
    uint8_t *flags = nullptr;
    uint32_t *pid = nullptr, *pid_prev = nullptr;
    double *wall_acc = nullptr, *wall_last = nullptr;
    uint32_t *tbits = nullptr;      // direct sweep: tiles that may hold non-bulk cells
    int *tile_lat = nullptr;        // batches: lattice of every sweep tile
    uint64_t *links = nullptr;      // per-cell link words (neighbour masks)
    uint32_t *nbody = nullptr;      // per-cell first neighbouring body
    uint32_t *near_list = nullptr;  // split direct sweep: compacted near-obstacle cells
    uint32_t *near_count = nullptr;
    uint32_t *chg = nullptr;        // re-mapping: cells whose owner changed this step
    uint32_t *chg_n = nullptr;
    bool split = false;             // direct sweep: near-obstacle cells in a kernel of their own
    int prefetch = 0;               // direct sweep: L2 prefetch of a later tile, bit p: sweeps of parity p
    __half *cl_par = nullptr;       // learned closure: FP16 network parameters
    bool closure = false;
    uint32_t *err = nullptr;
    uint32_t *tick = nullptr;       // step counter (advanced by the rigid-body kernel)

    int np = 0;
    PartDev P{};
    std::vector<void *> part_bufs;
    std::vector<int> shape_h;       // per body: LBM_SHAPE_*
    double *host_stage = nullptr;   // pinned: last F, M of every body (6 per body), then the error word
    std::vector<double> density_h;  // per body: density as given

    void *f_arena = nullptr;        // population allocation: guard | planes | guard
    long long guard = 0;            // guard band in elements on each side

    long long t = 0;
    int variant = SWEEP_DIRECT;     // sweep kernel variant
    int block = 128, grid = 0, ntiles = 0;
    int cpt = 1;                    // direct sweep: consecutive cells per thread (1, 2, 4)
    int remap_bpb = 8;
    // fused re-mapping step: launch form found by the probe (-1 not probed,
    // 0 unavailable, 1 cooperative, 2 cooperative + programmatic dependency),
    // user switch, grid and barrier state
    int remap_mode = -1;
    bool remap_fused = false;
    int remap_grid = 0;
    int np_pending = 0;             // bodies the launch shape was computed for
    GridBar *gbar = nullptr;
    // momentum stabilisation: sums and mean velocity (8 doubles), FP32 mean
    bool stab = false;
    double *stab_acc = nullptr;
    float *stab_accf = nullptr;

    bool graphs = true;
    cudaGraphExec_t gexec = nullptr;
    bool gvalid = false;
    long long graph_launches = 0;   // kernels in one replay of the two-step graph
    cudaGraphExec_t gexec1[2] = {nullptr, nullptr};  // one-step graphs, by parity of the step
    long long graph1_launches[2] = {0, 0};

    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double ms_acc = 0.0;
    long long timed_launches = 0;

    long long launches = 0;
    bool broken = false;
    std::string msg;
};

namespace {

// Makes the context's device current for the duration of a call and restores
// the caller's device afterwards (every entry point that takes a context).
struct DevGuard {
    int prev = -1;
    explicit DevGuard(const lbm_ctx *c) {
        if (!c) return;
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != c->device && cudaSetDevice(c->device) == cudaSuccess)
            prev = cur;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DevGuard(const DevGuard &) = delete;
    DevGuard &operator=(const DevGuard &) = delete;
};

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &m) {
    if (c) c->msg = m;
    return s;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void *dalloc(lbm_ctx *ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (ctx->dev_alloc) {
        p = ctx->dev_alloc(bytes, ctx->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dfree(lbm_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->dev_free)
        ctx->dev_free(p, ctx->user);
    else
        cudaFree(p);
}

void *owned_alloc(lbm_ctx *ctx, size_t bytes) {
    void *p = dalloc(ctx, bytes);
    if (p) {
        ctx->owned.push_back(p);
        ctx->device_bytes += bytes;
    }
    return p;
}

int storage_bytes(lbm_precision p) {
    switch (p) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16_OFFSET:
    case LBM_BF16_OFFSET: return 2;
    }
    return 0;
}

lbm_status check_desc(const lbm_grid_desc *d, std::string &m) {
    if (d->nx < 3 || d->ny < 3 || d->nz < 3) { m = "lattice sizes must be >= 3"; return LBM_ERR_ARG; }
    if ((long long)d->nx * d->ny * d->nz > 0x7FFFFFFFll) { m = "lattice above 2^31 cells"; return LBM_ERR_ARG; }
    if (!(d->tau > 0.5) || !std::isfinite(d->tau)) { m = "tau must be > 1/2"; return LBM_ERR_ARG; }
    if (!(d->magic > 0.0) || !std::isfinite(d->magic)) { m = "magic must be > 0"; return LBM_ERR_ARG; }
    if (!(d->rho0 > 0.0) || !std::isfinite(d->rho0)) { m = "rho0 must be > 0"; return LBM_ERR_ARG; }
    for (int a = 0; a < 3; ++a) {
        if (!(std::fabs(d->wall_u_lo[a]) < 0.1) || !(std::fabs(d->wall_u_hi[a]) < 0.1)) {
            m = "wall speed components must be below 0.1 (Mach limit)";
            return LBM_ERR_ARG;
        }
        if (!std::isfinite(d->body_force[a])) { m = "body force must be finite"; return LBM_ERR_ARG; }
    }
    if (storage_bytes(d->prec) == 0) { m = "unknown precision"; return LBM_ERR_ARG; }
    for (int a = 0; a < 3; ++a)
        if (d->free_slip[a] && d->periodic[a]) { m = "a free-slip axis cannot be periodic"; return LBM_ERR_ARG; }
    if (d->free_slip[1])
        for (int a = 0; a < 3; ++a)
            if (d->wall_u_lo[a] != 0.0 || d->wall_u_hi[a] != 0.0) {
                m = "free-slip y walls do not move";
                return LBM_ERR_ARG;
            }
    return LBM_OK;
}

int tile_cells(const lbm_ctx *ctx) { return ctx->variant == SWEEP_DIRECT ? ctx->block * ctx->cpt : STAGED_TILE; }

void fill_tiles(lbm_ctx *ctx) {
    int tile = 0;
    const int tc = tile_cells(ctx);
    for (auto &L : ctx->lat_h) {
        L.tile0 = tile;
        tile += (L.n + tc - 1) / tc;
    }
    ctx->ntiles = tile;
}

int default_grid(lbm_ctx *ctx) {
    if (ctx->variant == SWEEP_DIRECT) return ctx->ntiles > 0 ? ctx->ntiles : 1;  // one tile per block
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nb = sweep_max_active_blocks(ctx->prec, ctx->variant, ctx->block, ctx->cpt);
    if (nb <= 0) nb = 1;
    long long g = (long long)sms * nb;
    if (g > ctx->ntiles) g = ctx->ntiles;
    return (int)(g > 0 ? g : 1);
}

// Tiles ahead of its current one that a direct-sweep block prefetches: its
// own next tile on a persistent grid, else the tile one resident wave ahead
// (blocks start roughly in index order, so that tile's block starts about
// one block's duration later).
int prefetch_ahead(lbm_ctx *ctx) {
    if (ctx->grid < ctx->ntiles) return ctx->grid;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = sweep_max_active_blocks(ctx->prec, SWEEP_DIRECT, ctx->block, ctx->cpt);
    const long long w = (long long)(sms > 0 ? sms : 1) * (nb > 0 ? nb : 1);
    return (int)(w < ctx->ntiles ? w : ctx->ntiles);
}

SweepArgs sweep_args(lbm_ctx *ctx) {
    SweepArgs a;
    a.lat0 = ctx->lat_h[0];
    a.lat = ctx->lat_d;
    a.nlat = ctx->nlat;
    a.ntiles = ctx->ntiles;
    a.f = ctx->f;
    a.flags = ctx->flags;
    a.pid = ctx->pid;
    a.P = ctx->P;
    a.wall_acc = ctx->wall_acc;
    a.err = ctx->err;
    a.tbits = ctx->variant == SWEEP_DIRECT ? ctx->tbits : nullptr;
    a.tile_lat = ctx->tile_lat;
    a.links = ctx->links;
    a.nbody = ctx->nbody;
    a.tick = ctx->tick;
    const bool split = ctx->split && ctx->variant == SWEEP_DIRECT;
    const int ahead = ctx->variant == SWEEP_DIRECT && ctx->prefetch ? prefetch_ahead(ctx) : 0;
    a.pf_ahead[0] = (ctx->prefetch & 1) ? ahead : 0;
    a.pf_ahead[1] = (ctx->prefetch & 2) ? ahead : 0;
    a.near_list = split ? ctx->near_list : nullptr;
    a.near_count = split ? ctx->near_count : nullptr;
    return a;
}

// kernels one sweep issues (the split direct sweep: list, sweep, near cells)
int sweep_kernels(const lbm_ctx *ctx) { return (ctx->split && ctx->variant == SWEEP_DIRECT) ? 3 : 1; }

// Fused re-mapping launch: probed on first use; one resident wave at most,
// no more blocks than region units.
void update_remap_grid(lbm_ctx *ctx) {
    ctx->remap_grid = 0;
    if (!ctx->remap_fused || ctx->np_pending <= 0) return;
    if (ctx->remap_mode < 0) ctx->remap_mode = remap_fused_probe();
    const long long units = (long long)ctx->remap_bpb * ctx->np_pending;
    const long long wave = ctx->remap_mode > 0 ? remap_fused_max_blocks() : 0;
    ctx->remap_grid = (int)(units < wave ? units : wave);
}

bool fused_remap(const lbm_ctx *ctx) {
    return ctx->remap_fused && ctx->remap_mode > 0 && ctx->np > 0 && ctx->remap_grid > 0;
}

RemapArgs remap_args(lbm_ctx *ctx) {
    RemapArgs a;
    a.lat = ctx->lat_d;
    a.f = ctx->f;
    a.flags = ctx->flags;
    a.pid = ctx->pid;
    a.pid_prev = ctx->pid_prev;
    a.P = ctx->P;
    a.wall_acc = ctx->wall_acc;
    a.wall_last = ctx->wall_last;
    a.nlat = ctx->nlat;
    a.err = ctx->err;
    a.tbits = ctx->variant == SWEEP_DIRECT ? ctx->tbits : nullptr;
    a.tile = tile_cells(ctx);
    a.links = ctx->links;
    a.nbody = ctx->nbody;
    a.tick = ctx->tick;
    a.chg = ctx->chg;
    a.chg_n = ctx->chg_n;
    a.chg_cap = ctx->ncells;
    return a;
}

ClosureArgs closure_args(lbm_ctx *ctx) {
    ClosureArgs a{};
    a.lat = ctx->lat_d;
    a.f = ctx->f;
    a.flags = ctx->flags;
    a.P = ctx->P;
    a.feat = ctx->P.feat;
    return a;
}

MlpArgs closure_mlp_args(lbm_ctx *ctx) {
    MlpArgs m{};
    m.par16 = ctx->cl_par;
    m.x = ctx->P.feat;
    m.n = ctx->np;
    return m;
}

// Recount the direct sweep's tile bits from the flags (clears stale marks).
lbm_status recount_tiles(lbm_ctx *ctx) {
    if (ctx->variant != SWEEP_DIRECT) return LBM_OK;
    CK(launch_tile_bits(remap_args(ctx), ctx->ntiles, ctx->stream));
    ctx->launches += 1;
    return LBM_OK;
}

lbm_status upload_lattices(lbm_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->lat_d, ctx->lat_h.data(), sizeof(LatDev) * ctx->nlat, cudaMemcpyHostToDevice,
                       ctx->stream));
    if (ctx->tile_lat) CK(launch_tile_map(ctx->lat_d, ctx->nlat, ctx->ntiles, ctx->tile_lat, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

void drop_graph(lbm_ctx *ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gvalid = false;
    for (int p = 0; p < 2; ++p) {
        if (ctx->gexec1[p]) cudaGraphExecDestroy(ctx->gexec1[p]);
        ctx->gexec1[p] = nullptr;
    }
}

// One time step (Sec. 4.3): sweep at the parity of step t, rigid-body
// update, re-mapping for the parity of the next sweep.
lbm_status enqueue_step(lbm_ctx *ctx, bool timed) {
    const int parity = (int)(ctx->t & 1);
    SweepArgs sa = sweep_args(ctx);
    if (ctx->stab) {
        // mean fluid velocity of the state this sweep reads (Sec. 4.1)
        CK(launch_momentum_mean(ctx->prec, parity, ctx->lat_h[0], ctx->lat_d, ctx->f, ctx->flags, ctx->stab_acc,
                                ctx->stab_accf, ctx->stream));
        ctx->launches += 2;
    }
    if (timed) {
        if (ctx->ev_used + 2 > ctx->ev.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->ev.push_back(e);
            }
        }
        CK(cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream));
    }
    CK(launch_sweep(ctx->prec, parity, ctx->variant, sa, ctx->grid, ctx->block, ctx->cpt, ctx->stream));
    if (timed) {
        CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->stream));
        ctx->ev_used += 2;
        ctx->timed_launches += 1;
    }
    if (ctx->closure && ctx->np > 0) {
        // learned closure: features after the sweep, network, correction
        // added to the bodies' accumulators before their update
        const ClosureArgs ca = closure_args(ctx);
        CK(launch_closure_features(ctx->prec, 1 - parity, ca, ctx->stream));
        CK(launch_mlp_infer(closure_mlp_args(ctx), &ca, ctx->stream));
        ctx->launches += 2;
    }
    RemapArgs ra = remap_args(ctx);
    if (fused_remap(ctx)) {
        CK(launch_remap_fused(ctx->prec, 1 - parity, ra, ctx->remap_bpb, ctx->remap_grid, ctx->remap_mode,
                              ctx->gbar, ctx->stream));
        ctx->launches += sweep_kernels(ctx) + 1;
    } else {
        CK(launch_rigid_body(ra, ctx->stream));
        ctx->launches += sweep_kernels(ctx) + 1;
        if (ctx->np > 0) {
            CK(launch_remap_step(ctx->prec, 1 - parity, ra, ctx->remap_bpb, ctx->stream));
            ctx->launches += kernels_per_remap_step(ctx->np);
        }
    }
    ctx->t += 1;
    return LBM_OK;
}

lbm_status harvest_timing(lbm_ctx *ctx) {
    if (ctx->ev_used == 0) return LBM_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
        ctx->ms_acc += ms;
    }
    ctx->ev_used = 0;
    return LBM_OK;
}

lbm_status build_graph(lbm_ctx *ctx) {
    drop_graph(ctx);
    cudaGraph_t g = nullptr;
    const long long t0 = ctx->t, l0 = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    lbm_status s1 = enqueue_step(ctx, false);
    lbm_status s2 = s1 == LBM_OK ? enqueue_step(ctx, false) : s1;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->t = t0;
    ctx->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    if (s2 != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return s2;
    }
    if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->gexec = nullptr;
        return fail(ctx, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    ctx->gvalid = true;
    return LBM_OK;
}

// One step through the captured graph of its parity (built on first use): a
// caller that steps one at a time (and reads forces in between) pays one
// graph launch per step instead of one launch per kernel.
lbm_status graph_step(lbm_ctx *ctx) {
    const int par = (int)(ctx->t & 1);
    if (!ctx->gexec1[par]) {
        cudaGraph_t g = nullptr;
        const long long t0 = ctx->t, l0 = ctx->launches;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const lbm_status s1 = enqueue_step(ctx, false);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        ctx->t = t0;
        ctx->graph1_launches[par] = ctx->launches - l0;
        ctx->launches = l0;
        if (s1 != LBM_OK) {
            if (g) cudaGraphDestroy(g);
            return s1;
        }
        if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&ctx->gexec1[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->gexec1[par] = nullptr;
            return fail(ctx, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
    }
    CK(cudaGraphLaunch(ctx->gexec1[par], ctx->stream));
    ctx->t += 1;
    ctx->launches += ctx->graph1_launches[par];
    return LBM_OK;
}

lbm_status eval_err_word(lbm_ctx *ctx, uint32_t e) {
    if (e & ERR_NONFINITE) {
        ctx->broken = true;
        return fail(ctx, LBM_ERR_NUMERIC, "non-finite force, torque, particle state or wall momentum");
    }
    if (e & ERR_FSLIP_BODY) {
        ctx->broken = true;
        return fail(ctx, LBM_ERR_UNSUPPORTED, "a body reached the fluid layer next to a free-slip wall");
    }
    if (e & ERR_TIMEOUT) {
        ctx->broken = true;
        return fail(ctx, LBM_ERR_TIMEOUT, "device-side wait ran out");
    }
    return LBM_OK;
}

lbm_status check_err_word(lbm_ctx *ctx) {
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, ctx->err, sizeof(e), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return eval_err_word(ctx, e);
}

void free_particles(lbm_ctx *ctx) {
    for (void *p : ctx->part_bufs) {
        for (size_t i = 0; i < ctx->owned.size(); ++i)
            if (ctx->owned[i] == p) {
                ctx->owned.erase(ctx->owned.begin() + i);
                break;
            }
        dfree(ctx, p);
    }
    ctx->part_bufs.clear();
    ctx->P = PartDev{};
    ctx->np = 0;
}

// One particle buffer; a failed allocation raises *failed (the buffers
// allocated so far stay in part_bufs, so free_particles releases them).
template <class T>
T *part_alloc(lbm_ctx *ctx, size_t count, bool *failed) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    void *p = dalloc(ctx, bytes);
    if (p) {
        ctx->part_bufs.push_back(p);
        ctx->owned.push_back(p);
    } else {
        *failed = true;
    }
    return static_cast<T *>(p);
}

// Row-major rotation matrix of a unit quaternion (w,x,y,z); the same
// arithmetic order as the device mapping.
void quat_matrix_host(const double *q, double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

lbm_status create_common(const lbm_grid_desc *cells, int ncells, lbm_ctx **out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!cells || ncells <= 0) return LBM_ERR_ARG;
    std::string m;
    for (int i = 0; i < ncells; ++i) {
        lbm_status s = check_desc(&cells[i], m);
        if (s != LBM_OK) return s;
        if (cells[i].prec != cells[0].prec || cells[i].cuda_stream != cells[0].cuda_stream ||
            cells[i].dev_alloc != cells[0].dev_alloc || cells[i].dev_free != cells[0].dev_free)
            return LBM_ERR_ARG;
    }
    if ((cells[0].dev_alloc == nullptr) != (cells[0].dev_free == nullptr)) return LBM_ERR_ARG;
    lbm_ctx *ctx = new lbm_ctx();
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return LBM_ERR_CUDA;
    }
    ctx->prec = cells[0].prec;
    ctx->esize = storage_bytes(ctx->prec);
    ctx->stream = (cudaStream_t)cells[0].cuda_stream;
    ctx->dev_alloc = cells[0].dev_alloc;
    ctx->dev_free = cells[0].dev_free;
    ctx->user = cells[0].user;
    ctx->graphs = ctx->stream != nullptr;
    ctx->nlat = ncells;
    ctx->lat_h.resize(ncells);
    long long foff = 0, coff = 0;
    for (int i = 0; i < ncells; ++i) {
        const lbm_grid_desc &d = cells[i];
        LatDev &L = ctx->lat_h[i];
        memset(&L, 0, sizeof(L));
        L.nx = d.nx;
        L.ny = d.ny;
        L.nz = d.nz;
        L.n = d.nx * d.ny * d.nz;
        // planes start on 64-element (>= 128-byte) boundaries; LBM_PLANE_PAD
        // extra elements keep the 19 plane starts from sharing one DRAM
        // channel pattern when n is a large power of two
        L.npad = (L.n + 63) / 64 * 64 + LBM_PLANE_PAD;
        L.f_off = foff;
        L.c_off = coff;
        L.divx.init((uint32_t)d.nx);
        L.divxy.init((uint32_t)(d.nx * d.ny));
        L.px = d.periodic[0] ? 1 : 0;
        L.py = d.periodic[1] ? 1 : 0;
        L.pz = d.periodic[2] ? 1 : 0;
        L.fsx = d.free_slip[0] ? 1 : 0;
        L.fsy = d.free_slip[1] ? 1 : 0;
        L.fsz = d.free_slip[2] ? 1 : 0;
        L.omega = 1.0 / d.tau;
        L.omega_odd = 1.0 / (d.magic / (d.tau - 0.5) + 0.5);
        L.rho0 = d.rho0;
        L.inv_rho0 = 1.0 / d.rho0;
        L.rho18 = d.rho0 / 18.0;
        L.rho18f[0] = (float)L.rho18;
        L.rho18f[1] = (float)(L.rho18 - (double)L.rho18f[0]);
        for (int a = 0; a < 3; ++a) {
            L.wlo[a] = d.wall_u_lo[a];
            L.whi[a] = d.wall_u_hi[a];
            L.g[a] = d.body_force[a];
        }
        // learned closure scales: shear rate between moving y walls, viscosity
        L.cl_gamma = d.periodic[1] ? 0.0f : (float)(std::fabs(d.wall_u_hi[0] - d.wall_u_lo[0]) / (d.ny - 2.0));
        L.cl_mu = (float)(d.rho0 * (d.tau - 0.5) / 3.0);
        L.fomega = (float)L.omega;
        L.fomega_odd = (float)L.omega_odd;
        L.frho0 = (float)L.rho0;
        L.finv_rho0 = (float)L.inv_rho0;
        for (int a = 0; a < 3; ++a) {
            L.fg[a] = (float)L.g[a];
            L.fwlo[a] = (float)L.wlo[a];
            L.fwhi[a] = (float)L.whi[a];
        }
        for (int q = 0; q < Q; ++q) L.off[q] = cx(q) + cy(q) * d.nx + cz(q) * d.nx * d.ny;
        {
            // collision constants (see collide in the sweep)
            const double om = L.omega, oo = L.omega_odd, r0 = L.rho0, w1 = 1.0 / 18.0, w2 = 1.0 / 36.0;
            const double k[11] = {1.0 - om,           om / 3.0,           -1.5 * r0,          0.5 * (1.0 - om),
                                  0.5 * (1.0 - oo),   om * w1,            om * w2,            4.5 * r0 * om * w1,
                                  4.5 * r0 * om * w2, 3.0 * r0 * oo * w1, 3.0 * r0 * oo * w2};
            for (int i = 0; i < 11; ++i) {
                L.kd[i] = k[i];
                L.kf[i] = (float)k[i];
            }
            for (int i = 0; i < 9; ++i) {
                const int q = 2 * i + 1;
                const double cg = cx(q) * d.body_force[0] + cy(q) * d.body_force[1] + cz(q) * d.body_force[2];
                L.fsd[i] = 3.0 * wq(q) * r0 * cg;
                L.fsf[i] = (float)L.fsd[i];
            }
        }
        foff += (long long)Q * L.npad;
        coff += (L.n + 255) / 256 * 256;
        // a shifted staging window reaches at most nx*ny + nx + 1 cells (plus one
        // tile of slack) beyond its plane
        const long long reach = (long long)d.nx * d.ny + d.nx + 1 + 2 * STAGED_TILE;
        if (reach > ctx->guard) ctx->guard = reach;
    }
    ctx->guard = (ctx->guard + 63) / 64 * 64;
    ctx->f_elems = foff;
    ctx->ncells = coff;
    fill_tiles(ctx);

    ctx->lat_d = (LatDev *)owned_alloc(ctx, sizeof(LatDev) * ncells);
    ctx->f_arena = owned_alloc(ctx, (size_t)(foff + 2 * ctx->guard) * ctx->esize);
    ctx->f = ctx->f_arena ? (char *)ctx->f_arena + ctx->guard * ctx->esize : nullptr;
    ctx->flags = (uint8_t *)owned_alloc(ctx, (size_t)coff);
    ctx->pid = (uint32_t *)owned_alloc(ctx, (size_t)coff * 4);
    ctx->pid_prev = (uint32_t *)owned_alloc(ctx, (size_t)coff * 4);
    ctx->links = (uint64_t *)owned_alloc(ctx, (size_t)coff * 8);
    ctx->nbody = (uint32_t *)owned_alloc(ctx, (size_t)coff * 4);
    ctx->near_list = (uint32_t *)owned_alloc(ctx, (size_t)coff * 4);
    ctx->near_count = (uint32_t *)owned_alloc(ctx, 16);
    ctx->chg = (uint32_t *)owned_alloc(ctx, (size_t)coff * 4);
    ctx->chg_n = (uint32_t *)owned_alloc(ctx, 16);
    ctx->wall_acc = (double *)owned_alloc(ctx, sizeof(double) * 6 * ACC_COPIES * ncells);
    ctx->wall_last = (double *)owned_alloc(ctx, sizeof(double) * 6 * ncells);
    ctx->err = (uint32_t *)owned_alloc(ctx, 16);
    ctx->tick = (uint32_t *)owned_alloc(ctx, 16);
    ctx->gbar = (GridBar *)owned_alloc(ctx, 16);
    ctx->stab_acc = (double *)owned_alloc(ctx, 64);
    ctx->stab_accf = (float *)owned_alloc(ctx, 16);
    {
        long long tiles32 = 0;  // tiles of the smallest direct-sweep tile (32 cells)
        for (auto &L : ctx->lat_h) tiles32 += (L.n + 31) / 32;
        ctx->tbits = (uint32_t *)owned_alloc(ctx, sizeof(uint32_t) * (size_t)(tiles32 / 32 + 1));
        if (ncells > 1) ctx->tile_lat = (int *)owned_alloc(ctx, sizeof(int) * (size_t)(tiles32 + 1));
    }
    if (!ctx->lat_d || !ctx->f || !ctx->flags || !ctx->pid || !ctx->pid_prev || !ctx->wall_acc ||
        !ctx->wall_last || !ctx->err || !ctx->tick || !ctx->tbits || !ctx->links || !ctx->nbody || !ctx->near_list ||
        !ctx->near_count || !ctx->chg || !ctx->chg_n || !ctx->gbar || !ctx->stab_acc || !ctx->stab_accf || (ncells > 1 && !ctx->tile_lat)) {
        lbm_destroy(ctx);
        return LBM_ERR_OOM;
    }
    lbm_status s = upload_lattices(ctx);
    if (s != LBM_OK) {
        lbm_destroy(ctx);
        return s;
    }
    // fluid at rest: every stored offset f - w rho0 is zero
    if (cudaMemsetAsync(ctx->f_arena, 0, (size_t)(foff + 2 * ctx->guard) * ctx->esize, ctx->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(ctx->flags, 0, (size_t)coff, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->pid, 0xFF, (size_t)coff * 4, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->wall_acc, 0, sizeof(double) * 6 * ACC_COPIES * ncells, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->wall_last, 0, sizeof(double) * 6 * ncells, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->err, 0, 16, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->tick, 0, 16, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->chg_n, 0, 16, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->gbar, 0, 16, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->stab_acc, 0, 64, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->stab_accf, 0, 16, ctx->stream) != cudaSuccess) {
        lbm_destroy(ctx);
        return LBM_ERR_CUDA;
    }
    for (int i = 0; i < ncells; ++i) {
        if (launch_init_cells(ctx->lat_h[i], ctx->lat_d + i, ctx->flags, ctx->pid, ctx->pid_prev, ctx->links,
                              ctx->nbody,
                              ctx->stream) != cudaSuccess) {
            lbm_destroy(ctx);
            return LBM_ERR_CUDA;
        }
        ctx->launches += 2;
    }
    ctx->grid = default_grid(ctx);
    if (recount_tiles(ctx) != LBM_OK || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        lbm_destroy(ctx);
        return LBM_ERR_CUDA;
    }
    *out = ctx;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_grid_desc *desc, lbm_ctx **out) { return create_common(desc, 1, out); }

lbm_status lbm_create_batch(const lbm_grid_desc *cells, int ncells, lbm_ctx **out) {
    return create_common(cells, ncells, out);
}

lbm_status lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    for (void *p : ctx->owned) dfree(ctx, p);
    if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
    delete ctx;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->msg.c_str() : "null context"; }

const char *lbm_status_string(lbm_status s) {
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_STATE: return "invalid state";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_NUMERIC: return "non-finite value";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

lbm_status lbm_set_particles(lbm_ctx *ctx, const lbm_particle *p, int n) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (n < 0 || (n > 0 && !p)) return fail(ctx, LBM_ERR_ARG, "bad particle array");
    // validate and derive host-side quantities
    std::vector<double> pos(3 * n), quat(4 * n), vel(3 * n), om(3 * n), L(3 * n), semi(3 * n), mass(n),
        inertia(3 * n), extF(3 * n), extM(3 * n), minv(n), Iinv(3 * n), R64(9 * (size_t)n);
    std::vector<float> bodyf(BF_STRIDE * (size_t)n, 0.0f);
    std::vector<int> cell(n), fixed(n), region(6 * n), shape(n);
    std::vector<double> density(n);
    for (int i = 0; i < n; ++i) {
        const lbm_particle &b = p[i];
        if (b.cell < 0 || b.cell >= ctx->nlat) return fail(ctx, LBM_ERR_ARG, "particle cell index out of range");
        if (!(b.semi_axes[0] > 0 && b.semi_axes[1] > 0 && b.semi_axes[2] > 0))
            return fail(ctx, LBM_ERR_ARG, "semi-axes must be positive");
        if (!(b.density > 0)) return fail(ctx, LBM_ERR_ARG, "density must be positive");
        if (b.shape != LBM_SHAPE_ELLIPSOID && b.shape != LBM_SHAPE_SPHEROCYLINDER)
            return fail(ctx, LBM_ERR_ARG, "unknown particle shape");
        const bool capsule = b.shape == LBM_SHAPE_SPHEROCYLINDER;
        if (capsule && !(b.semi_axes[1] == b.semi_axes[2] && b.semi_axes[0] >= b.semi_axes[1]))
            return fail(ctx, LBM_ERR_ARG, "spherocylinder needs semi_axes = (L/2, r, r) with L/2 >= r");
        double q[4] = {b.quat[0], b.quat[1], b.quat[2], b.quat[3]};
        const double nrm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(nrm > 0) || !std::isfinite(nrm)) return fail(ctx, LBM_ERR_ARG, "quaternion must be non-zero");
        for (int k = 0; k < 4; ++k) q[k] /= nrm;
        const LatDev &Lt = ctx->lat_h[b.cell];
        double R[9];
        quat_matrix_host(q, R);
        const int dims[3] = {Lt.nx, Lt.ny, Lt.nz}, per[3] = {Lt.px, Lt.py, Lt.pz};
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(b.pos[a]) || !std::isfinite(b.vel[a]) || !std::isfinite(b.omega[a]))
                return fail(ctx, LBM_ERR_ARG, "non-finite particle state");
            // half extent along a: ellipsoid sqrt(sum_j (R_aj s_j)^2),
            // spherocylinder |R_a0| (L/2 - r) + r
            const double s0 = capsule ? b.semi_axes[1] : b.semi_axes[0];
            const double e0 = R[3 * a] * s0, e1 = R[3 * a + 1] * b.semi_axes[1], e2 = R[3 * a + 2] * b.semi_axes[2];
            const double h = std::sqrt(e0 * e0 + e1 * e1 + e2 * e2) +
                             (capsule ? std::fabs(R[3 * a]) * (b.semi_axes[0] - b.semi_axes[1]) : 0.0);
            if (!per[a] && (b.pos[a] - h < 1.0 || b.pos[a] + h > dims[a] - 2.0))
                return fail(ctx, LBM_ERR_ARG, "particle not inside the fluid region");
            const int fsl = a == 0 ? Lt.fsx : (a == 1 ? Lt.fsy : Lt.fsz);
            if (fsl && (b.pos[a] - h < 1.5 || b.pos[a] + h > dims[a] - 2.5))
                return fail(ctx, LBM_ERR_ARG, "particle on the fluid layer next to a free-slip wall");
            if (per[a] && !(b.pos[a] >= 0.0 && b.pos[a] < dims[a]))
                return fail(ctx, LBM_ERR_ARG, "periodic coordinate outside [0, n)");
            int lo = (int)std::floor(b.pos[a] - h) - 2, hi = (int)std::ceil(b.pos[a] + h) + 2;
            if (per[a]) {
                if (hi - lo + 1 > dims[a]) { lo = 0; hi = dims[a] - 1; }
            } else {
                lo = lo < 0 ? 0 : lo;
                hi = hi > dims[a] - 1 ? dims[a] - 1 : hi;
            }
            region[6 * i + a] = lo;
            region[6 * i + 3 + a] = hi - lo + 1;
        }
        double m, I[3];
        if (capsule) {
            // cylinder of length 2h (mass mc) and a sphere of radius r split
            // into the two end caps (mass ms); transverse moment of the caps by
            // the parallel-axis theorem (cap centroid 3r/8 from its flat face)
            const double r = b.semi_axes[1], h = b.semi_axes[0] - b.semi_axes[1];
            const double mc = b.density * M_PI * r * r * (2.0 * h);
            const double ms = b.density * (4.0 / 3.0) * M_PI * r * r * r;
            m = mc + ms;
            I[0] = mc * r * r / 2.0 + 2.0 * ms * r * r / 5.0;
            I[1] = mc * (r * r / 4.0 + (2.0 * h) * (2.0 * h) / 12.0) + ms * (2.0 * r * r / 5.0 + h * h + 3.0 * h * r / 4.0);
            I[2] = I[1];
        } else {
            const double A = b.semi_axes[0], B = b.semi_axes[1], Cc = b.semi_axes[2];
            m = b.density * (4.0 / 3.0) * M_PI * A * B * Cc;
            I[0] = m * (B * B + Cc * Cc) / 5.0;
            I[1] = m * (A * A + Cc * Cc) / 5.0;
            I[2] = m * (A * A + B * B) / 5.0;
        }
        // angular momentum L = R I R^T omega
        double ob[3], Lw[3];
        for (int a = 0; a < 3; ++a)
            ob[a] = (R[a] * b.omega[0] + R[3 + a] * b.omega[1] + R[6 + a] * b.omega[2]) * I[a];
        for (int a = 0; a < 3; ++a) Lw[a] = R[3 * a] * ob[0] + R[3 * a + 1] * ob[1] + R[3 * a + 2] * ob[2];
        for (int a = 0; a < 3; ++a) {
            pos[3 * i + a] = b.pos[a];
            vel[3 * i + a] = b.vel[a];
            om[3 * i + a] = b.omega[a];
            L[3 * i + a] = Lw[a];
            semi[3 * i + a] = b.semi_axes[a];
            inertia[3 * i + a] = I[a];
            extF[3 * i + a] = b.ext_force[a];
            extM[3 * i + a] = b.ext_torque[a];
        }
        for (int k = 0; k < 4; ++k) quat[4 * i + k] = q[k];
        mass[i] = m;
        minv[i] = 1.0 / m;
        for (int a = 0; a < 3; ++a) Iinv[3 * i + a] = 1.0 / I[a];
        for (int k = 0; k < 9; ++k) R64[9 * (size_t)i + k] = R[k];
        float *bf = &bodyf[BF_STRIDE * (size_t)i];
        for (int k = 0; k < 9; ++k) bf[BF_R + k] = (float)R[k];
        bf[BF_SHAPE] = capsule ? 1.0f : 0.0f;
        bf[BF_TUBE_H] = (float)(b.semi_axes[0] + 2.0);
        bf[BF_TUBE_R] = (float)(std::fmax(b.semi_axes[1], b.semi_axes[2]) + 2.0);
        bf[BF_CAPH] = capsule ? (float)((b.semi_axes[0] - b.semi_axes[1]) / b.semi_axes[1]) : 0.0f;
        for (int a = 0; a < 3; ++a) {
            bf[BF_INV + a] = (float)(1.0 / (capsule ? b.semi_axes[1] : b.semi_axes[a]));
            bf[BF_POS + a] = (float)b.pos[a];
            bf[BF_POSLO + a] = (float)(b.pos[a] - (double)bf[BF_POS + a]);
            bf[BF_U + a] = (float)b.vel[a];
            bf[BF_W + a] = (float)b.omega[a];
        }
        cell[i] = b.cell;
        fixed[i] = b.fixed ? 1 : 0;
        shape[i] = b.shape;
        density[i] = b.density;
    }
    // re-mapping launch shape: about four box cells per thread for the
    // largest body, at most ~16 blocks per SM over all bodies (with many
    // small bodies a block per body: each block first loads its body's
    // record, a cost paid once per block)
    {
        double amax = 0.0;
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) amax = std::fmax(amax, p[i].semi_axes[a]);
        const double side = 2.0 * amax + 7.0;
        const double vol = side * side * side;
        long long bpb = (long long)std::ceil(vol / (256.0 * 4.0));
        bpb = bpb < 1 ? 1 : (bpb > 1024 ? 1024 : bpb);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long cap = (long long)(sms > 0 ? sms : 1) * 16;
        if (n > 0 && bpb * n > cap) bpb = cap / n > 0 ? cap / n : 1;
        ctx->remap_bpb = (int)bpb;
        ctx->np_pending = n;
        update_remap_grid(ctx);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    free_particles(ctx);
    PartDev &P = ctx->P;
    P.np = n;
    const size_t m = n > 0 ? n : 1;
    bool failed = false;
    P.pos = part_alloc<double>(ctx, 3 * m, &failed);
    P.quat = part_alloc<double>(ctx, 4 * m, &failed);
    P.vel = part_alloc<double>(ctx, 3 * m, &failed);
    P.om = part_alloc<double>(ctx, 3 * m, &failed);
    P.L = part_alloc<double>(ctx, 3 * m, &failed);
    P.semi = part_alloc<double>(ctx, 3 * m, &failed);
    P.mass = part_alloc<double>(ctx, m, &failed);
    P.inertia = part_alloc<double>(ctx, 3 * m, &failed);
    P.minv = part_alloc<double>(ctx, m, &failed);
    P.Iinv = part_alloc<double>(ctx, 3 * m, &failed);
    P.bodyf = part_alloc<float>(ctx, BF_STRIDE * m, &failed);
    P.R64 = part_alloc<double>(ctx, 9 * m, &failed);
    P.feat = part_alloc<float>(ctx, (size_t)CL_IN * m, &failed);
    P.extF = part_alloc<double>(ctx, 3 * m, &failed);
    P.extM = part_alloc<double>(ctx, 3 * m, &failed);
    P.cell = part_alloc<int>(ctx, m, &failed);
    P.fixed = part_alloc<int>(ctx, m, &failed);
    P.pos_old = part_alloc<double>(ctx, 3 * m, &failed);
    P.vel_old = part_alloc<double>(ctx, 3 * m, &failed);
    P.om_old = part_alloc<double>(ctx, 3 * m, &failed);
    P.quat_old = part_alloc<double>(ctx, 4 * m, &failed);
    P.acc = part_alloc<double>(ctx, 6 * ACC_COPIES * m, &failed);
    P.last = part_alloc<double>(ctx, 6 * m, &failed);
    P.region = part_alloc<int>(ctx, 6 * m, &failed);
    P.changed = part_alloc<int>(ctx, m, &failed);
    if (failed) {
        // the previous bodies' cells are still mapped: map the lattices
        // without bodies, so that the context stays consistent (and usable)
        free_particles(ctx);
        if (n > 0) {
            const std::string keep = "particle buffers: device allocation failed";
            lbm_status s0 = lbm_set_particles(ctx, nullptr, 0);
            if (s0 != LBM_OK) ctx->broken = true;
            return fail(ctx, LBM_ERR_OOM, keep);
        }
        ctx->broken = true;
        return fail(ctx, LBM_ERR_OOM, "particle buffers: device allocation failed");
    }
    ctx->np = n;
    if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
    ctx->host_stage = nullptr;
    CK(cudaMallocHost((void **)&ctx->host_stage, sizeof(double) * (6 * m + 2)));
    ctx->shape_h = shape;
    ctx->density_h = density;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
    };
    CK(up(P.pos, pos.data(), 8 * pos.size()));
    CK(up(P.quat, quat.data(), 8 * quat.size()));
    CK(up(P.vel, vel.data(), 8 * vel.size()));
    CK(up(P.om, om.data(), 8 * om.size()));
    CK(up(P.L, L.data(), 8 * L.size()));
    CK(up(P.semi, semi.data(), 8 * semi.size()));
    CK(up(P.mass, mass.data(), 8 * mass.size()));
    CK(up(P.inertia, inertia.data(), 8 * inertia.size()));
    CK(up(P.minv, minv.data(), 8 * minv.size()));
    CK(up(P.Iinv, Iinv.data(), 8 * Iinv.size()));
    CK(up(P.bodyf, bodyf.data(), 4 * bodyf.size()));
    CK(up(P.R64, R64.data(), 8 * R64.size()));
    CK(up(P.extF, extF.data(), 8 * extF.size()));
    CK(up(P.extM, extM.data(), 8 * extM.size()));
    CK(up(P.cell, cell.data(), 4 * cell.size()));
    CK(up(P.fixed, fixed.data(), 4 * fixed.size()));
    CK(up(P.pos_old, pos.data(), 8 * pos.size()));
    CK(up(P.vel_old, vel.data(), 8 * vel.size()));
    CK(up(P.om_old, om.data(), 8 * om.size()));
    CK(up(P.quat_old, quat.data(), 8 * quat.size()));
    CK(up(P.region, region.data(), 4 * region.size()));
    CK(cudaMemsetAsync(P.acc, 0, sizeof(double) * 6 * ACC_COPIES * m, ctx->stream));
    CK(cudaMemsetAsync(P.last, 0, sizeof(double) * 6 * m, ctx->stream));
    CK(cudaMemsetAsync(P.changed, 0, sizeof(int) * m, ctx->stream));
    // full re-map of every lattice for the next sweep's parity
    RemapArgs ra = remap_args(ctx);
    const int next_odd = (int)(ctx->t & 1);
    for (int li = 0; li < ctx->nlat; ++li) CK(launch_clear_particles(ctx->lat_h[li], ra, li, ctx->stream));
    CK(launch_claim_all(ra, ctx->remap_bpb, ctx->stream));
    for (int li = 0; li < ctx->nlat; ++li)
        CK(launch_remap_full(ctx->prec, next_odd, ra, ctx->lat_h[li], li, ctx->stream));
    ctx->launches += 3 * ctx->nlat + (n > 0 ? 1 : 0);
    lbm_status st = recount_tiles(ctx);
    if (st != LBM_OK) return st;
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int nsteps) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (nsteps < 0) return fail(ctx, LBM_ERR_ARG, "nsteps < 0");
    if (ctx->broken) return fail(ctx, LBM_ERR_STATE, "context stopped after an earlier error");
    int left = nsteps;
    // the direct sweep's tile bits are recounted every 64 steps (moving
    // bodies leave marked tiles behind; a stale mark only costs time)
    const bool moving = ctx->np > 0 && ctx->variant == SWEEP_DIRECT;
    auto maybe_recount = [&]() -> lbm_status {
        return (moving && (ctx->t & 63) == 0) ? recount_tiles(ctx) : LBM_OK;
    };
    const bool use_graph = ctx->graphs && !ctx->timing && ctx->stream != nullptr;
    if (use_graph && left >= 1) {
        if (ctx->t & 1) {
            lbm_status s = graph_step(ctx);
            if (s == LBM_OK) s = maybe_recount();
            if (s != LBM_OK) return s;
            --left;
        }
        if (left >= 2) {
            if (!ctx->gvalid) {
                lbm_status s = build_graph(ctx);
                if (s != LBM_OK) return s;
            }
            while (left >= 2) {
                CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
                ctx->t += 2;
                ctx->launches += ctx->graph_launches;
                left -= 2;
                lbm_status s = maybe_recount();
                if (s != LBM_OK) return s;
            }
        }
        if (left == 1) {
            lbm_status s = graph_step(ctx);
            if (s == LBM_OK) s = maybe_recount();
            if (s != LBM_OK) return s;
            --left;
        }
    }
    while (left > 0) {
        lbm_status s = enqueue_step(ctx, ctx->timing);
        if (s == LBM_OK) s = maybe_recount();
        if (s != LBM_OK) return s;
        --left;
    }
    if (ctx->timing && ctx->ev_used > 4096) return harvest_timing(ctx);
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *ctx) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    return check_err_word(ctx);
}

lbm_status lbm_get_forces(lbm_ctx *ctx, double *force3n, double *torque3n, int n) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (n < 0 || n > ctx->np) return fail(ctx, LBM_ERR_ARG, "n out of range");
    if (n == 0) return LBM_OK;
    // forces and the error word into pinned memory, one synchronisation
    double *buf = ctx->host_stage;
    uint32_t *err = reinterpret_cast<uint32_t *>(buf + 6 * (size_t)ctx->np);
    CK(cudaMemcpyAsync(buf, ctx->P.last, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(err, ctx->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (force3n) force3n[3 * i + a] = buf[6 * i + a];
            if (torque3n) torque3n[3 * i + a] = buf[6 * i + 3 + a];
        }
    return eval_err_word(ctx, *err);
}

lbm_status lbm_get_wall_forces(lbm_ctx *ctx, int cell, double *f6) {
    if (!ctx || !f6) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (cell < 0 || cell >= ctx->nlat) return fail(ctx, LBM_ERR_ARG, "cell out of range");
    CK(cudaMemcpyAsync(f6, ctx->wall_last + 6 * cell, sizeof(double) * 6, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_get_particles(lbm_ctx *ctx, lbm_particle *p, int n) {
    if (!ctx || (n > 0 && !p)) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (n < 0 || n > ctx->np) return fail(ctx, LBM_ERR_ARG, "n out of range");
    if (n == 0) return LBM_OK;
    std::vector<double> pos(3 * n), quat(4 * n), vel(3 * n), om(3 * n), semi(3 * n), mass(n), eF(3 * n), eM(3 * n);
    std::vector<int> cell(n), fixed(n);
    const PartDev &P = ctx->P;
    CK(cudaMemcpyAsync(pos.data(), P.pos, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(quat.data(), P.quat, 32 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(vel.data(), P.vel, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(om.data(), P.om, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(semi.data(), P.semi, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(mass.data(), P.mass, 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(eF.data(), P.extF, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(eM.data(), P.extM, 24 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(cell.data(), P.cell, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(fixed.data(), P.fixed, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < n; ++i) {
        lbm_particle &b = p[i];
        for (int a = 0; a < 3; ++a) {
            b.pos[a] = pos[3 * i + a];
            b.vel[a] = vel[3 * i + a];
            b.omega[a] = om[3 * i + a];
            b.semi_axes[a] = semi[3 * i + a];
            b.ext_force[a] = eF[3 * i + a];
            b.ext_torque[a] = eM[3 * i + a];
        }
        for (int k = 0; k < 4; ++k) b.quat[k] = quat[4 * i + k];
        b.density = ctx->density_h[i];
        b.cell = cell[i];
        b.fixed = fixed[i];
        b.shape = ctx->shape_h[i];
    }
    return LBM_OK;
}

lbm_status lbm_set_external(lbm_ctx *ctx, const double *force3n, const double *torque3n, int n) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (n < 0 || n > ctx->np) return fail(ctx, LBM_ERR_ARG, "n out of range");
    if (n == 0) return LBM_OK;
    if (force3n) CK(cudaMemcpyAsync(ctx->P.extF, force3n, 24 * n, cudaMemcpyHostToDevice, ctx->stream));
    if (torque3n) CK(cudaMemcpyAsync(ctx->P.extM, torque3n, 24 * n, cudaMemcpyHostToDevice, ctx->stream));
    // pageable host memory: the copy has been staged when cudaMemcpyAsync returns
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_ctx *ctx, int cell, double *rho, double *u3, uint8_t *flags, uint32_t *pid,
                          double *pdfs) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (cell < 0 || cell >= ctx->nlat) return fail(ctx, LBM_ERR_ARG, "cell out of range");
    const LatDev &h = ctx->lat_h[cell];
    const size_t n = h.n;
    const size_t bytes = (rho ? 8 * n : 0) + (u3 ? 24 * n : 0) + (pdfs ? 8 * Q * n : 0) + (flags ? n : 0) + 64;
    char *scratch = (char *)dalloc(ctx, bytes);
    if (!scratch) return fail(ctx, LBM_ERR_OOM, "field scratch");
    double *d_rho = nullptr, *d_u = nullptr, *d_pdfs = nullptr;
    uint8_t *d_fl = nullptr;
    size_t off = 0;
    if (rho) { d_rho = (double *)(scratch + off); off += 8 * n; }
    if (u3) { d_u = (double *)(scratch + off); off += 24 * n; }
    if (pdfs) { d_pdfs = (double *)(scratch + off); off += 8 * Q * n; }
    if (flags) { d_fl = (uint8_t *)(scratch + off); off += n; }
    lbm_status st = LBM_OK;
    cudaError_t e = launch_canonical(ctx->prec, (int)(ctx->t & 1), h, ctx->lat_d + cell, ctx->f, ctx->flags,
                                     ctx->pid, d_rho, d_u, d_fl, d_pdfs, ctx->stream);
    ctx->launches += 1;
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, d_rho, 8 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && u3) e = cudaMemcpyAsync(u3, d_u, 24 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && pdfs) e = cudaMemcpyAsync(pdfs, d_pdfs, 8 * Q * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && flags) e = cudaMemcpyAsync(flags, d_fl, n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && pid)
        e = cudaMemcpyAsync(pid, ctx->pid + h.c_off, 4 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = fail(ctx, LBM_ERR_CUDA, std::string("get_fields: ") + cudaGetErrorString(e));
    dfree(ctx, scratch);
    return st;
}

lbm_status lbm_set_pdfs(lbm_ctx *ctx, int cell, const double *pdfs) {
    if (!ctx || !pdfs) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (cell < 0 || cell >= ctx->nlat) return fail(ctx, LBM_ERR_ARG, "cell out of range");
    const LatDev &h = ctx->lat_h[cell];
    const size_t bytes = 8 * Q * (size_t)h.n;
    double *d = (double *)dalloc(ctx, bytes);
    if (!d) return fail(ctx, LBM_ERR_OOM, "pdf scratch");
    cudaError_t e = cudaMemcpyAsync(d, pdfs, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = launch_set_pdfs(ctx->prec, (int)(ctx->t & 1), h, ctx->lat_d + cell, ctx->f, ctx->flags, d, ctx->stream);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d);
    if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string("set_pdfs: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Link compaction without device allocation.  The per-block link counts that
// lbm_get_links keeps in freshly allocated scratch live here in one fixed
// array in device memory, present on every GPU that loads this library until
// the process exits.  Host code must not pass the array's name to a kernel:
// on the host that name is only a stand-in, not a device address.  Its
// device address is looked up once per device, with that device current.
// ---------------------------------------------------------------------------
namespace {

constexpr int LINKS_NOALLOC_MAX_BLOCKS = 65536;  // 65536 tiles of 256 cells
static __device__ __align__(256) int g_links_scratch[LINKS_NOALLOC_MAX_BLOCKS];

constexpr int MAX_DEVICES = 64;
std::mutex g_links_scratch_mu;
int *g_links_scratch_addr[MAX_DEVICES] = {};

// Device address of g_links_scratch on the current device (looked up on the
// first call for that device).  Every entry point runs with its context's
// device current, so this is the address on the context's device.
cudaError_t links_scratch_address(int **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_links_scratch_mu);
    if (!g_links_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_links_scratch);
        if (e != cudaSuccess) return e;
        g_links_scratch_addr[dev] = static_cast<int *>(p);
    }
    *out = g_links_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

lbm_status lbm_get_links_noalloc(lbm_ctx *ctx, int cell, int32_t *d_idx, int8_t *d_q, uint32_t *d_pid, int cap,
                                 int *d_count) {
    if (!ctx || !d_count || cap < 0) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (cell < 0 || cell >= ctx->nlat) return fail(ctx, LBM_ERR_ARG, "cell out of range");
    const LatDev &h = ctx->lat_h[cell];
    const int nblocks = (h.n + 255) / 256;
    if (nblocks > LINKS_NOALLOC_MAX_BLOCKS)
        return fail(ctx, LBM_ERR_ARG,
                    "lattice larger than the allocation-free link scratch (at most 16777216 cells)");
    int *scratch = nullptr;
    CK(links_scratch_address(&scratch));
    // every one of the nblocks entries is written by the count pass before the
    // scan reads it, so nothing left by an earlier call needs clearing
    CK(launch_links(h, ctx->lat_d + cell, ctx->flags, ctx->pid, scratch, nblocks, cap ? d_idx : nullptr,
                    cap ? d_q : nullptr, cap ? d_pid : nullptr, cap, d_count, ctx->stream));
    ctx->launches += 3;
    return LBM_OK;
}

lbm_status lbm_get_links(lbm_ctx *ctx, int cell, int32_t *idx, int8_t *q, uint32_t *pid, int cap, int *count) {
    if (!ctx || !count || cap < 0) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (cell < 0 || cell >= ctx->nlat) return fail(ctx, LBM_ERR_ARG, "cell out of range");
    const LatDev &h = ctx->lat_h[cell];
    const int nblocks = (h.n + 255) / 256;
    const size_t cap_sz = cap > 0 ? (size_t)cap : 0;
    const size_t bytes = 4 * (size_t)nblocks + 16 + cap_sz * (4 + 4 + 1) + 64;
    char *scratch = (char *)dalloc(ctx, bytes);
    if (!scratch) return fail(ctx, LBM_ERR_OOM, "link scratch");
    int *bc = (int *)scratch;
    int *total = bc + nblocks;
    int32_t *d_idx = (int32_t *)(scratch + 4 * (size_t)nblocks + 16);
    uint32_t *d_pid = (uint32_t *)(d_idx + cap_sz);
    int8_t *d_q = (int8_t *)(d_pid + cap_sz);
    cudaError_t e = launch_links(h, ctx->lat_d + cell, ctx->flags, ctx->pid, bc, nblocks, cap ? d_idx : nullptr,
                                 cap ? d_q : nullptr, cap ? d_pid : nullptr, cap, total, ctx->stream);
    ctx->launches += 3;
    int tot = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, total, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    const int nw = tot < cap ? tot : cap;
    if (e == cudaSuccess && nw > 0 && idx) e = cudaMemcpyAsync(idx, d_idx, 4 * (size_t)nw, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && nw > 0 && q) e = cudaMemcpyAsync(q, d_q, (size_t)nw, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && nw > 0 && pid) e = cudaMemcpyAsync(pid, d_pid, 4 * (size_t)nw, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, scratch);
    if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string("get_links: ") + cudaGetErrorString(e));
    *count = tot;
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *info) {
    if (!ctx || !info) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    long long n = 0;
    for (auto &L : ctx->lat_h) n += L.n;
    info->ncells_total = n;
    info->nfluid_hint = -1;
    info->nlattices = ctx->nlat;
    info->nparticles = ctx->np;
    info->steps_done = ctx->t;
    info->device_bytes = ctx->device_bytes;
    info->sweep_grid = ctx->grid;
    info->sweep_block = ctx->variant == SWEEP_RING ? 0 : (ctx->variant == SWEEP_STAGED ? -1 : ctx->block);
    info->bytes_per_population = ctx->esize;
    info->sweep_split = (ctx->split && ctx->variant == SWEEP_DIRECT) ? 1 : 0;
    info->remap_fused = fused_remap(ctx) ? 1 : 0;
    info->remap_grid = fused_remap(ctx) ? ctx->remap_grid : 0;
    info->cells_per_thread = ctx->variant == SWEEP_DIRECT ? ctx->cpt : 1;
    info->device = ctx->device;
    info->sweep_prefetch = ctx->variant == SWEEP_DIRECT && ctx->prefetch ? prefetch_ahead(ctx) : 0;
    info->sweep_prefetch_mode = ctx->variant != SWEEP_DIRECT ? LBM_PREFETCH_OFF
                                : ctx->prefetch == 3         ? LBM_PREFETCH_ALL
                                : ctx->prefetch == 1         ? LBM_PREFETCH_EVEN
                                : ctx->prefetch == 2         ? LBM_PREFETCH_ODD
                                                             : LBM_PREFETCH_OFF;
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_ctx *ctx, int block, int grid) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (block != 0 && block != -1 && (block < 32 || block > 256 || block % 32))
        return fail(ctx, LBM_ERR_ARG, "block must be 0 (ring sweep), -1 (staged sweep) or a multiple of 32 in [32, 256]");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->variant = block == 0 ? SWEEP_RING : (block == -1 ? SWEEP_STAGED : SWEEP_DIRECT);
    ctx->block = block <= 0 ? STAGED_TILE : block;
    fill_tiles(ctx);
    lbm_status s = upload_lattices(ctx);
    if (s != LBM_OK) return s;
    ctx->grid = grid > 0 ? (grid < ctx->ntiles ? grid : ctx->ntiles) : default_grid(ctx);
    drop_graph(ctx);
    s = recount_tiles(ctx);  // the tile size may have changed
    if (s != LBM_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_set_cells_per_thread(lbm_ctx *ctx, int cpt) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (!sweep_cpt_supported(ctx->prec, cpt))
        return fail(ctx, LBM_ERR_ARG, "cells per thread must be 1, 2 or 4 (1 or 2 for FP64 storage)");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->cpt = cpt;
    fill_tiles(ctx);
    lbm_status s = upload_lattices(ctx);
    if (s != LBM_OK) return s;
    ctx->grid = default_grid(ctx);
    drop_graph(ctx);
    s = recount_tiles(ctx);  // the tile size changes with the cells per thread
    if (s != LBM_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx *ctx, int *block_out, int *grid_out) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    // back up the populations; sweeps below run on the live buffers
    const size_t fbytes = (size_t)ctx->f_elems * ctx->esize;
    void *backup = dalloc(ctx, fbytes);
    if (!backup) return fail(ctx, LBM_ERR_OOM, "autotune backup");
    CK(cudaMemcpyAsync(backup, ctx->f, fbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // candidates: the ring sweep (block 0), the staged sweep (block -1) and
    // the direct sweep at two block sizes with 1, 2 or 4 cells per thread,
    // fused or split, each with persistent grids (1x, 2x resident) and one
    // tile per block; the direct sweep's L2 prefetch is chosen for the even-
    // and the odd-step sweeps on their own (each timed with and without it)
    struct Cand {
        int block, cpt;
        bool split;
    };
    std::vector<Cand> cands = {{0, 1, false}, {-1, 1, false}};
    for (int blk : {128, 256})
        for (int c : {1, 2, 4})
            if (sweep_cpt_supported(ctx->prec, c))
                for (bool sp : {false, true}) cands.push_back({blk, c, sp});
    double best = 1e30;
    int bb = ctx->variant == SWEEP_RING ? 0 : (ctx->variant == SWEEP_STAGED ? -1 : ctx->block);
    int bg = ctx->grid, bc = ctx->cpt;
    bool bsplit = ctx->split;
    int bpf = ctx->prefetch;
    constexpr int REPS = 4;
    cudaEvent_t ev[2 * REPS + 1];
    for (cudaEvent_t &e : ev) CK(cudaEventCreate(&e));
    for (const Cand &cand : cands) {
        ctx->cpt = cand.cpt;
        lbm_status s = lbm_set_launch(ctx, cand.block, 0);
        if (s != LBM_OK) break;
        ctx->split = cand.split;
        const int occ = sweep_max_active_blocks(ctx->prec, ctx->variant, ctx->block, ctx->cpt);
        if (occ <= 0) continue;
        const int grids[] = {sms * occ, 2 * sms * occ, ctx->ntiles};
        for (int gr : grids) {
            if (gr > ctx->ntiles) gr = ctx->ntiles;
            ctx->grid = gr;
            // ms[pf][parity]: summed over REPS sweeps of that parity
            float ms[2][2] = {{0.f, 0.f}, {1e30f, 1e30f}};
            for (int pf = 0; pf < (ctx->variant == SWEEP_DIRECT ? 2 : 1); ++pf) {
                ctx->prefetch = pf ? 3 : 0;
                SweepArgs sa = sweep_args(ctx);
                for (int w = 0; w < 2; ++w) {
                    CK(launch_sweep(ctx->prec, 0, ctx->variant, sa, gr, ctx->block, ctx->cpt, ctx->stream));
                    CK(launch_sweep(ctx->prec, 1, ctx->variant, sa, gr, ctx->block, ctx->cpt, ctx->stream));
                }
                CK(cudaEventRecord(ev[0], ctx->stream));
                for (int r = 0; r < REPS; ++r) {
                    CK(launch_sweep(ctx->prec, 0, ctx->variant, sa, gr, ctx->block, ctx->cpt, ctx->stream));
                    CK(cudaEventRecord(ev[2 * r + 1], ctx->stream));
                    CK(launch_sweep(ctx->prec, 1, ctx->variant, sa, gr, ctx->block, ctx->cpt, ctx->stream));
                    CK(cudaEventRecord(ev[2 * r + 2], ctx->stream));
                }
                CK(cudaEventSynchronize(ev[2 * REPS]));
                ctx->launches += 2 * (2 + REPS) * sweep_kernels(ctx);
                ms[pf][0] = ms[pf][1] = 0.f;
                for (int k = 0; k < 2 * REPS; ++k) {
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
                    ms[pf][k & 1] += t;
                }
            }
            const int pe = ms[1][0] < ms[0][0] ? 1 : 0, po = ms[1][1] < ms[0][1] ? 1 : 0;
            const double total = (double)ms[pe][0] + ms[po][1];
            if (total < best) {
                best = total;
                bb = cand.block;
                bg = gr;
                bc = cand.cpt;
                bsplit = ctx->split;
                bpf = pe | (po << 1);
            }
        }
    }
    for (cudaEvent_t &e : ev) cudaEventDestroy(e);
    ctx->split = bsplit;
    ctx->prefetch = bpf;
    ctx->cpt = bb > 0 ? bc : 1;
    lbm_status s = lbm_set_launch(ctx, bb, bg);
    CK(cudaMemcpyAsync(ctx->f, backup, fbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->np > 0) CK(cudaMemsetAsync(ctx->P.acc, 0, sizeof(double) * 6 * ACC_COPIES * ctx->np, ctx->stream));
    CK(cudaMemsetAsync(ctx->wall_acc, 0, sizeof(double) * 6 * ACC_COPIES * ctx->nlat, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, backup);
    if (block_out) *block_out = bb;
    if (grid_out) *grid_out = bg;
    return s;
}

lbm_status lbm_set_sweep_split(lbm_ctx *ctx, int enable) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->split = enable != 0;
    drop_graph(ctx);
    return LBM_OK;
}

lbm_status lbm_set_sweep_prefetch(lbm_ctx *ctx, int mode) {
    if (!ctx) return LBM_ERR_ARG;
    if (mode < LBM_PREFETCH_OFF || mode > LBM_PREFETCH_ODD)
        return fail(ctx, LBM_ERR_ARG, "prefetch mode must be one of LBM_PREFETCH_OFF/ALL/EVEN/ODD");
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prefetch = mode == LBM_PREFETCH_ALL ? 3 : mode == LBM_PREFETCH_EVEN ? 1 : mode == LBM_PREFETCH_ODD ? 2 : 0;
    drop_graph(ctx);
    return LBM_OK;
}

lbm_status lbm_set_momentum_stabilisation(lbm_ctx *ctx, int enable) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (ctx->nlat != 1) return fail(ctx, LBM_ERR_UNSUPPORTED, "momentum stabilisation needs a single lattice");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stab = enable != 0;
    ctx->lat_h[0].ubar = ctx->stab ? ctx->stab_acc + 4 : nullptr;
    ctx->lat_h[0].ubarf = ctx->stab ? ctx->stab_accf : nullptr;
    CK(cudaMemsetAsync(ctx->stab_acc, 0, 64, ctx->stream));
    CK(cudaMemsetAsync(ctx->stab_accf, 0, 16, ctx->stream));
    lbm_status st = upload_lattices(ctx);
    drop_graph(ctx);
    return st;
}

lbm_status lbm_set_remap_fused(lbm_ctx *ctx, int enable) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->remap_fused = enable != 0;
    update_remap_grid(ctx);
    drop_graph(ctx);
    return LBM_OK;
}

lbm_status lbm_set_wait_limit(lbm_ctx *ctx, unsigned polls) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpyAsync(&ctx->gbar->limit, &polls, sizeof(unsigned), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status lbm_set_graphs(lbm_ctx *ctx, int enable) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    ctx->graphs = enable != 0 && ctx->stream != nullptr;
    if (!ctx->graphs) drop_graph(ctx);
    return LBM_OK;
}

lbm_status lbm_set_sweep_timing(lbm_ctx *ctx, int enable) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    lbm_status s = harvest_timing(ctx);
    if (s != LBM_OK) return s;
    ctx->timing = enable != 0;
    ctx->ms_acc = 0.0;
    ctx->timed_launches = 0;
    return LBM_OK;
}

lbm_status lbm_get_sweep_timing(lbm_ctx *ctx, double *ms, long long *launches) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    lbm_status s = harvest_timing(ctx);
    if (s != LBM_OK) return s;
    if (ms) *ms = ctx->ms_acc;
    if (launches) *launches = ctx->timed_launches;
    ctx->ms_acc = 0.0;
    ctx->timed_launches = 0;
    return LBM_OK;
}

lbm_status lbm_get_launch_count(lbm_ctx *ctx, long long *launches) {
    if (!ctx || !launches) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    *launches = ctx->launches;
    return LBM_OK;
}

lbm_status lbm_set_closure(lbm_ctx *ctx, const void *params, size_t bytes) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);  // the captured step changes with the closure
    if (!params) {
        ctx->closure = false;
        return LBM_OK;
    }
    if (bytes != sizeof(__half) * CL_PARAMS)
        return fail(ctx, LBM_ERR_ARG, "closure parameters must be LBM_CLOSURE_PARAMS half values");
    if (!ctx->cl_par) {
        ctx->cl_par = (__half *)owned_alloc(ctx, sizeof(__half) * CL_PARAMS);
        if (!ctx->cl_par) return fail(ctx, LBM_ERR_OOM, "closure parameters");
    }
    CK(cudaMemcpyAsync(ctx->cl_par, params, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->closure = true;
    return LBM_OK;
}

lbm_status lbm_closure_features(lbm_ctx *ctx, float *features, int n) {
    if (!ctx) return LBM_ERR_ARG;
    DevGuard dg(ctx);
    if (n != ctx->np || (n > 0 && !features)) return fail(ctx, LBM_ERR_ARG, "n must equal the number of bodies");
    if (n == 0) return LBM_OK;
    CK(launch_closure_features(ctx->prec, (int)(ctx->t & 1), closure_args(ctx), ctx->stream));
    ctx->launches += 1;
    CK(cudaMemcpyAsync(features, ctx->P.feat, sizeof(float) * CL_IN * (size_t)n, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

}  // extern "C"
