// teuk_api.cu -- the C ABI of include/teuk.h: argument validation, device memory
// (stream-ordered allocation on the caller's stream), kernel launches and copies.
// No arithmetic of the time step happens on the host.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "teuk.h"
#include "teuk_aux.cuh"
#include "teuk_internal.cuh"
#include "teuk_step_common.cuh"

using namespace teuk;

namespace {

constexpr double kPi = 3.141592653589793238462643;

// The launch configuration a per-step graph captured (compared byte for byte).
struct StepGraphKey {
    InstDev d;
    const int* part;
    int strip;
    int pad;
};

struct Instance {
    teuk_params p{};
    double drs = 0, dth = 0, dt = 0, rp = 0, rm = 0;
    int pitch = 0;
    int64_t step = 0;   // time level of the state
    int cur = 0;        // buffer holding the state
    void* state[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    size_t plane_bytes = 0;
    void* coef_h = nullptr;
    void* coef_i = nullptr;
    double* x_int = nullptr;
    double* x_half = nullptr;
    RTab2* rtab = nullptr;      // [nr] (half node, node) per column (FP32 paths)
    ThTab* thtab = nullptr;     // [nth]
    // source
    bool src_on = false;
    teuk_orbit orbit{};
    double rs0 = 0, sig_r = 0, sig_t = 0, drs0_dr0 = 0;
    double2* P_win = nullptr;   // P_int | P_half | dP_int | dP_half | Q_int | Q_half
                                // (moving particle: Q_int | Q_half only)
    double* amps = nullptr;
    void* traj_buf = nullptr;   // moving particle: samples | amp | gr | gt (SourceDev)
    SourceDev sd{};
    // waveform ring: time levels [wave_lo, wave_hi) are held
    double2* wave = nullptr;
    int64_t wave_cap = 0, wave_lo = 0, wave_hi = 0;
    int i_e = 0;
    double f_e = 0, r_ext = 0;
    int strip = 0;      // r* columns per work item chosen for this instance (0 = context default)
    int resident = 0;   // blocks of its step kernel the GPU holds at once
    double* stage = nullptr;    // u-layout staging of set/get_state, allocated on first use
    // column partition of the per-step launch for strip length part_strip (see
    // refresh_partition); d_part holds n_rstar ints
    int* d_part = nullptr;
    std::vector<int> h_part;
    int part_strip = 0;
    int fault_col = -1;         // testing aid (teuk_set_fill_fault)
    // slab of a larger grid (teuk_params.slab_ncols > 0): local column k is grid column
    // k + off; local columns 0 and n_rstar - 1 are halos (or the grid's own ends)
    int off = 0;
    bool slab = false;
    bool ext_here = true;       // the extraction radius lies between two local columns
    // resident launches (teuk_set_resident): halo h (0 = off), plan, exchange slots and
    // flags (nb + 1 ints: the blocks' flags, then the abort flag)
    int res_h = 0;
    int res_bps = 1;
    bool res_blocked = false;   // blocked launches: h steps a launch, no exchange (teuk_set_blocked)
    ResidentPlan res_plan;
    unsigned char* res_xg = nullptr;
    int* res_flags = nullptr;
    // per-step launches replayed from CUDA graphs of kStepGraph steps (one graph per parity
    // of the buffer holding the state); sg_key is the launch configuration each captured
    int64_t* d_step = nullptr;      // the graphs' step base (device)
    int64_t graph_base = -1;        // the step *d_step holds (-1: unknown)
    int64_t h_step = 0;             // host source of the base's copy
    cudaGraphExec_t sg_exec[2] = {nullptr, nullptr};
    StepGraphKey sg_key[2] = {};
    bool sg_failed = false;         // capture refused (legacy stream): launch directly
};

// Device side of the batched persistent launch of one context: one persistent kernel
// per block-size class (instances whose theta pitch is the same), run one after the
// other (classes are independent).
struct BatchClass {
    int pitch = 0;                  // threads per block
    std::vector<int> members;       // instance indices
    size_t off = 0;                 // descriptor offset in the blob
    unsigned long long* d_counter = nullptr;
    int* d_flags = nullptr;
    int64_t flags_cap = 0;
    int64_t items = -1;
    int grid = 0;
    int max_nth = 0;
    bool moving = false;            // a member has a moving particle
    BatchDev bd{};
};

struct Batch {
    bool alloc = false;
    char* d_blob = nullptr;         // descriptors of the current call, all classes
    size_t blob_bytes = 0;
    int* d_abort = nullptr;
    std::vector<BatchClass> cls;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
};

}  // namespace

namespace {
// Device memory of a context: stream-ordered cudaMallocAsync / cudaFreeAsync on the
// context's stream, or the caller's allocator (teuk_set_allocator) in force when the
// context was created.
struct DevAlloc {
    teuk_alloc_fn alloc = nullptr;
    teuk_free_fn free = nullptr;
    void* user = nullptr;
    cudaError_t get(void** p, size_t bytes, cudaStream_t s) const {
        if (!alloc) return cudaMallocAsync(p, bytes, s);
        *p = alloc(bytes, (void*)s, user);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    void put(void* p, cudaStream_t s) const {
        if (!p) return;
        if (free) free(p, (void*)s, user);
        else cudaFreeAsync(p, s);
    }
};
DevAlloc g_alloc;   // the allocator new contexts take (teuk_set_allocator)
}  // namespace

struct teuk_ctx {
    DevAlloc al;
    cudaStream_t stream = nullptr;
    int prec = 0;
    std::vector<Instance> inst;
    unsigned* status = nullptr;
    std::string err;
    int strip = 0;           // r* columns per thread block (0 = automatic)
    int steps_per_launch = 1;
    int64_t launches = 0;
    Batch batch;
    int64_t inject_skip_item = -1;   // testing aid: a work item that never releases its flag
    long long spin_limit = 20000000LL;
    double2* sum_buf = nullptr;      // teuk_extract's summed records, grown on demand
    int64_t sum_cap = 0;
    cudaStream_t cap = nullptr;      // private stream on which the context's CUDA graphs are
                                     // captured (any stream, the legacy one included, can
                                     // then replay them)
};

static std::string g_create_err = "no error";

namespace teuk {
// Error text for calls that have no context (returned by teuk_last_error(NULL)).
void set_global_error(const std::string& msg) { g_create_err = msg; }
}  // namespace teuk

template <class T>
static cudaError_t dmalloc(const teuk_ctx* c, T** p, size_t bytes, cudaStream_t s) {
    return c->al.get((void**)p, bytes, s);
}
static void dfree(const teuk_ctx* c, void* p, cudaStream_t s) { c->al.put(p, s); }

#define TK_FAIL(ctx, code, ...)                                              \
    do {                                                                     \
        char _b[512];                                                        \
        snprintf(_b, sizeof(_b), __VA_ARGS__);                               \
        (ctx)->err = _b;                                                     \
        return code;                                                         \
    } while (0)

#define TK_CUDA(ctx, call)                                                   \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) {                                             \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(_e); \
            return _e == cudaErrorMemoryAllocation ? TEUK_ENOMEM : TEUK_ECUDA; \
        }                                                                    \
    } while (0)

namespace {

double rstar_of_r(double M, double a, double r) {
    double d = std::sqrt(M * M - a * a), rp = M + d, rm = M - d;
    double k = 2.0 * M / (rp - rm);
    return r + k * rp * std::log((r - rp) / (2.0 * M)) - k * rm * std::log((r - rm) / (2.0 * M));
}

// Validate one instance and fill its derived geometry.  Returns an error text or "".
std::string derive(const teuk_params& p, Instance& I) {
    if (!(p.M > 0) || !(std::fabs(p.a) < p.M)) return "need M > 0 and |a| < M";
    if (p.n_rstar < 8) return "n_rstar must be >= 8";
    if (p.n_theta < 4 || p.n_theta > 1024) return "n_theta must be in [4, 1024]";
    if ((int64_t)p.n_rstar * p.n_theta > (int64_t)1 << 30) return "grid too large";
    if (!(p.rstar_max > p.rstar_min)) return "need rstar_max > rstar_min";
    if (p.prec < 0 || p.prec > 3)
        return "prec must be TEUK_FP64, TEUK_FP32, TEUK_FP32_KAHAN or TEUK_FP64_DF";
    if (p.wave_capacity < 0) return "wave_capacity must be >= 0";
    I.p = p;
    I.drs = (p.rstar_max - p.rstar_min) / (double)(p.n_rstar - 1);
    I.dth = kPi / (double)p.n_theta;
    double d = std::sqrt(p.M * p.M - p.a * p.a);
    I.rp = p.M + d;
    I.rm = p.M - d;
    if (p.dt > 0) {
        I.dt = p.dt;
    } else if (p.dt_rule == 0) {
        I.dt = p.courant * I.drs;
    } else if (p.dt_rule == 1) {
        double lim = I.dth / (double)(std::abs(p.m) + std::abs(p.s) + 2);
        I.dt = p.courant * std::fmin(I.drs, lim);
    } else {
        return "dt_rule must be 0 or 1";
    }
    if (!(I.dt > 0) || !std::isfinite(I.dt)) return "time step must be positive";
    double pos = (p.rstar_ext - p.rstar_min) / I.drs;
    if (!(pos >= 0.0) || !(pos <= (double)(p.n_rstar - 1))) return "rstar_ext outside the grid";
    int ie = (int)std::floor(pos);
    if (ie > p.n_rstar - 2) ie = p.n_rstar - 2;
    I.i_e = ie;
    I.f_e = (p.rstar_ext - (p.rstar_min + ie * I.drs)) / I.drs;
    if (p.slab_ncols < 0) return "slab_ncols must be >= 0";
    if (p.slab_ncols > 0) {
        // the owned grid columns [col0, col0 + ncols), all interior, plus one halo per side
        if (p.slab_col0 < 1 || p.slab_ncols < 2 || p.slab_col0 + p.slab_ncols > p.n_rstar - 1)
            return "a slab must own >= 2 interior columns: 1 <= slab_col0, slab_col0 + slab_ncols <= n_rstar - 1";
        I.slab = true;
        I.off = p.slab_col0 - 1;
        I.p.n_rstar = p.slab_ncols + 2;
        I.i_e = ie - I.off;
        I.ext_here = I.i_e >= 0 && I.i_e <= I.p.n_rstar - 2;
        if (!I.ext_here) {
            I.i_e = 0;
            I.f_e = 0.0;
        }
    }
    I.pitch = (p.n_theta + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
    I.wave_cap = p.wave_capacity > 0 ? p.wave_capacity : 4096;
    return "";
}

InstDev dev_of(const teuk_ctx* c, const Instance& I) {
    InstDev d{};
    d.nr = I.p.n_rstar;
    d.nth = I.p.n_theta;
    d.pitch = I.pitch;
    d.prec = I.p.prec;
    d.drs = I.drs;
    d.dth = I.dth;
    d.dt = I.dt;
    // pole rule of Sec. 2.2 (stated for s = -2) by the parity of |m + s|: the pole
    // behaviour theta^|m+s| of the spin-weighted harmonics, the paper's rule for even s
    d.ghost = (std::abs(I.p.m + I.p.s) % 2 == 0) ? 1.0 : -1.0;
    d.ghost_f = (float)d.ghost;
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 2; ++k) d.buf[b][k] = I.state[b][k];
    d.coef_h = I.coef_h;
    d.coef_i = I.coef_i;
    d.rtab = I.rtab;
    d.thtab = I.thtab;
    d.src = I.sd;
    d.src.on = I.src_on ? 1 : 0;
    d.i_e = I.i_e;
    d.f_e = I.f_e;
    d.wave = I.wave;
    d.wave_cap = I.wave_cap;
    d.status = c->status;
    d.fault_col = I.fault_col;
    return d;
}

// Strip length so that the grid holds about 16 warps per SM on 152 SMs, at least
// 8 columns (a strip reads 2 columns beyond its outputs).
// Strip length that gives one wave of resident blocks (at most 512 columns).  Grids too
// small to fill the GPU get one column per block: the step time is then the ring's
// start-up plus the strip, so the shortest strip is fastest (800 x 64 on GB300: 4.2 us
// per step at one column, 8.2 us at eight).
int auto_strip(const Instance& I) {
    int64_t blocks = I.resident > 0 ? I.resident : 1;
    int64_t cols = I.p.n_rstar - 2;
    int64_t L = (cols + blocks - 1) / blocks;
    if (L < 1) L = 1;
    if (L > 512) L = 512;
    return (int)L;
}

int eff_strip(const teuk_ctx* c, const Instance& I) {
    int L = I.strip > 0 ? I.strip : (c->strip > 0 ? c->strip : auto_strip(I));
    return std::max(1, std::min(L, I.p.n_rstar - 2));
}

// Column partition of the per-step launch: the same number of blocks as uniform strips
// of the effective length, cut so that the blocks have about equal cost.  A column costs
// 1, a column of the source window 1 + alpha (its source terms) and the extraction
// column 2 more (the FP64 waveform record).  alpha, measured on GB300 (16384 x 256 step
// time against alpha): FP32 paths 0.25, FP64 0.1, double-float 0.4; for a moving
// particle, whose source terms also carry the per-step Gaussian factors, FP32 0.8 and
// double-float 0.6 (FP64: no better value than 0.1).  Without it the blocks holding the source window
// finish last and every step waits for them.  Built on the host whenever the strip
// length or the source changes, so a step never allocates or copies.
teuk_status refresh_partition(teuk_ctx* c, Instance& I) {
    const int strip = eff_strip(c, I);
    const int nr = I.p.n_rstar;
    const int nb = (nr - 2 + strip - 1) / strip;
    const double alpha = I.p.prec == TEUK_FP64      ? 0.1
                         : I.p.prec == TEUK_FP64_DF ? (I.sd.moving ? 0.6 : 0.4)
                                                    : (I.sd.moving ? 0.8 : 0.25);
    int wlo = nr, whi = 0;
    if (I.src_on) {
        wlo = std::min(I.sd.i_lo, I.sd.h_lo + 1);
        whi = std::max(I.sd.i_lo + I.sd.ni, I.sd.h_lo + I.sd.nh + 1);
    }
    std::vector<double> cum(nr, 0.0);  // cum[col] = cost of the columns 1 .. col-1
    for (int col = 2; col <= nr - 1; ++col) {
        const int q = col - 1;
        cum[col] = cum[col - 1] + 1.0 + ((q >= wlo && q < whi) ? alpha : 0.0) + (q == I.i_e ? 2.0 : 0.0);
    }
    const double total = cum[nr - 1];
    I.h_part.assign(nb + 1, 0);
    I.h_part[0] = 1;
    I.h_part[nb] = nr - 1;
    int col = 1;
    for (int k = 1; k < nb; ++k) {
        const double t = total * k / nb;
        const int lo = I.h_part[k - 1] + 1, hi = nr - 1 - (nb - k);
        col = std::max(col, lo);
        while (col < hi && cum[col + 1] <= t) ++col;
        if (col < hi && t - cum[col] > cum[col + 1] - t) ++col;
        I.h_part[k] = col;
    }
    if (!I.d_part) TK_CUDA(c, dmalloc(c, (void**)&I.d_part, sizeof(int) * nr, c->stream));
    // (from pageable memory: staged before the call returns, so h_part may change after)
    TK_CUDA(c, cudaMemcpyAsync(I.d_part, I.h_part.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice,
                               c->stream));
    I.part_strip = strip;
    return TEUK_OK;
}

teuk_status refresh_partitions(teuk_ctx* c) {
    for (Instance& I : c->inst) {
        teuk_status st = refresh_partition(c, I);
        if (st) return st;
    }
    return TEUK_OK;
}

// The 2D coefficient tables [9][n_rstar][pitch] at half and integer nodes, in the
// instance's precision: read by the FP64 and double-float step kernels and their adjoint,
// built at creation.  FP32 instances form their coefficients from 1D tables, forward and
// adjoint, and have none.
teuk_status coef_tables(teuk_ctx* c, Instance& I) {
    if (I.coef_h) return TEUK_OK;
    const teuk_params& q = I.p;
    const size_t cs = q.prec == TEUK_FP64 ? sizeof(double) : q.prec == TEUK_FP64_DF ? sizeof(float2) : sizeof(float);
    const size_t cbytes = (size_t)kNCoef * q.n_rstar * I.pitch * cs;
    TK_CUDA(c, dmalloc(c, &I.coef_h, cbytes, c->stream));
    TK_CUDA(c, dmalloc(c, &I.coef_i, cbytes, c->stream));
    launch_coefficients(c->stream, q.prec, q.M, q.a, q.s, q.m, q.rstar_min, I.drs, I.dth, I.dt,
                        q.n_rstar, q.n_theta, I.pitch, I.x_int, I.x_half, I.coef_h, I.coef_i);
    c->launches++;
    TK_CUDA(c, cudaGetLastError());
    return TEUK_OK;
}

void do_step(teuk_ctx* c, Instance& I, int strip) {
    launch_step(c->stream, dev_of(c, I), I.step, I.cur, strip, I.part_strip == strip ? I.d_part : nullptr);
    c->launches++;
    I.cur = 1 - I.cur;
    I.step++;
}

void do_extract(teuk_ctx* c, Instance& I) {
    launch_extract(c->stream, dev_of(c, I), I.step, I.cur);
    c->launches++;
}

// The private capture stream (created on first use; nullptr if that fails).
cudaStream_t capture_stream(teuk_ctx* c) {
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap = nullptr;
    }
    return c->cap;
}

// Steps per replayed graph (even, so that the state returns to the buffer it started in).
constexpr int64_t kStepGraph = 64;

// The graph of kStepGraph per-step launches of the descriptor dv (the instance's own,
// or one whose buffers or records are elsewhere) starting in buffer p, captured on first
// use and again whenever the descriptor or configuration changed (one cached graph per
// starting buffer).  The graph is captured on the context's private stream and replayed
// on its stream (any stream, the legacy default one included).  Returns nullptr while
// the caller is capturing the context's stream, or if capture failed; the steps are
// then launched directly.
cudaGraphExec_t step_graph_of(teuk_ctx* c, Instance& I, const InstDev& dv, int p, int strip,
                              const int* part) {
    if (I.sg_failed) return nullptr;
    cudaStreamCaptureStatus ucs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &ucs) != cudaSuccess || ucs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    if (!I.d_step && dmalloc(c, (void**)&I.d_step, sizeof(int64_t), c->stream) != cudaSuccess) {
        cudaGetLastError();
        I.sg_failed = true;
        return nullptr;
    }
    // (object representations copied byte for byte, so that the comparison below sees
    // only the members)
    StepGraphKey key;
    std::memset(&key, 0, sizeof key);
    std::memcpy(&key.d, &dv, sizeof dv);
    key.d.step_base = I.d_step;
    key.part = part;
    key.strip = strip;
    if (I.sg_exec[p] && std::memcmp(&key, &I.sg_key[p], sizeof key) == 0) return I.sg_exec[p];
    if (I.sg_exec[p]) cudaGraphExecDestroy(I.sg_exec[p]);
    I.sg_exec[p] = nullptr;
    cudaGraph_t g = nullptr;
    cudaStream_t cs = capture_stream(c);
    if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        I.sg_failed = true;
        return nullptr;
    }
    for (int64_t k = 0; k < kStepGraph; ++k)
        launch_step(cs, key.d, k, (int)((p + k) & 1), strip, key.part);
    launch_advance_step(cs, I.d_step, kStepGraph);
    cudaGraphExec_t e = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g ||
        cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        I.sg_failed = true;
        return nullptr;
    }
    cudaGraphDestroy(g);
    I.sg_exec[p] = e;
    std::memcpy(&I.sg_key[p], &key, sizeof key);
    return e;
}

cudaGraphExec_t step_graph(teuk_ctx* c, Instance& I, int strip) {
    return step_graph_of(c, I, dev_of(c, I), I.cur, strip, I.part_strip == strip ? I.d_part : nullptr);
}

// Run count steps of the descriptor dv from buffer cur at time level `level` on stream st:
// whole graphs of kStepGraph steps (the device step base set to `level` first), then
// the rest one launch at a time.  Returns the buffer holding the result.
int run_steps(teuk_ctx* c, Instance& I, const InstDev& dv, cudaStream_t st, int cur, int64_t level,
              int64_t count, int strip) {
    const int* part = I.part_strip == strip ? I.d_part : nullptr;
    int64_t k = 0;
    cudaGraphExec_t e = (st == c->stream && count >= kStepGraph)
                            ? step_graph_of(c, I, dv, cur, strip, part) : nullptr;
    if (e && I.graph_base != level) {
        I.h_step = level;
        if (cudaMemcpyAsync(I.d_step, &I.h_step, sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
        } else {
            I.graph_base = level;
        }
    }
    if (e)
        for (; k + kStepGraph <= count; k += kStepGraph) {
            if (cudaGraphLaunch(e, st) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            c->launches += kStepGraph + 1;
            I.graph_base += kStepGraph;   // advanced by the graph's last node
        }
    for (; k < count; ++k) {   // (kStepGraph is even: the graphs leave the buffer unchanged)
        launch_step(st, dv, level + k, cur, strip, part);
        c->launches++;
        cur = 1 - cur;
    }
    return cur;
}

void free_instance(const teuk_ctx* c, Instance& I) {
    const cudaStream_t s = c->stream;
    for (int p = 0; p < 2; ++p)
        if (I.sg_exec[p]) cudaGraphExecDestroy(I.sg_exec[p]);
    if (I.d_step) dfree(c, I.d_step, s);
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 2; ++k)
            if (I.state[b][k]) dfree(c, I.state[b][k], s);
    void* ptrs[] = {I.coef_h, I.coef_i, I.x_int, I.x_half, I.P_win, I.amps, I.wave, I.rtab, I.thtab,
                    I.stage, I.d_part, I.traj_buf, I.res_xg, I.res_flags};
    for (void* q : ptrs)
        if (q) dfree(c, q, s);
    I = Instance();
}

teuk_status check_instance(teuk_ctx* c, int instance) {
    if (!c) return TEUK_EINVAL;
    if (instance < 0 || instance >= (int)c->inst.size())
        TK_FAIL(c, TEUK_EINVAL, "instance %d out of range [0, %d)", instance, (int)c->inst.size());
    return TEUK_OK;
}

}  // namespace

// ------------------------------------------------------------------ create

extern "C" teuk_status teuk_create(const teuk_params* p, int n_instances, void* cuda_stream,
                                   teuk_ctx** out) {
    if (out) *out = nullptr;
    if (!p || !out || n_instances < 1) {
        g_create_err = "teuk_create: null argument or n_instances < 1";
        return TEUK_EINVAL;
    }
    std::vector<Instance> inst(n_instances);
    for (int k = 0; k < n_instances; ++k) {
        std::string e = derive(p[k], inst[k]);
        if (!e.empty()) {
            g_create_err = "instance " + std::to_string(k) + ": " + e;
            return TEUK_EINVAL;
        }
        if (p[k].prec != p[0].prec) {
            g_create_err = "all instances of a context must use the same precision";
            return TEUK_EINVAL;
        }
    }
    int dev = -1;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) {
        g_create_err = std::string("no usable CUDA device: ") + cudaGetErrorString(ce);
        return TEUK_ECUDA;
    }
    teuk_ctx* c = new teuk_ctx();
    c->al = g_alloc;
    c->stream = (cudaStream_t)cuda_stream;
    c->prec = p[0].prec;
    c->inst = std::move(inst);
    auto fail = [&](teuk_status st) {
        g_create_err = c->err;
        teuk_destroy(c);
        return st;
    };
#define TK_CCUDA(call)                                                            \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            c->err = std::string(#call) + ": " + cudaGetErrorString(_e);          \
            return fail(_e == cudaErrorMemoryAllocation ? TEUK_ENOMEM : TEUK_ECUDA); \
        }                                                                         \
    } while (0)
    TK_CCUDA(prepare_step_kernels());
    for (Instance& I : c->inst) I.resident = step_resident_blocks((int)I.p.prec, I.pitch);
    TK_CCUDA(dmalloc(c, (void**)&c->status, sizeof(unsigned), c->stream));
    TK_CCUDA(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    for (Instance& I : c->inst) {
        const teuk_params& q = I.p;
        size_t es = q.prec == TEUK_FP64 ? sizeof(double2) : sizeof(float4);
        int nplanes = q.prec == TEUK_FP32 ? 1 : 2;
        I.plane_bytes = (size_t)q.n_rstar * I.pitch * es;
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < nplanes; ++k) {
                TK_CCUDA(dmalloc(c, &I.state[b][k], I.plane_bytes, c->stream));
                TK_CCUDA(cudaMemsetAsync(I.state[b][k], 0, I.plane_bytes, c->stream));
            }
        TK_CCUDA(dmalloc(c, (void**)&I.x_int, sizeof(double) * q.n_rstar, c->stream));
        TK_CCUDA(dmalloc(c, (void**)&I.x_half, sizeof(double) * q.n_rstar, c->stream));
        TK_CCUDA(dmalloc(c, (void**)&I.wave, sizeof(double2) * I.wave_cap * q.n_theta,
                                 c->stream));
        launch_invert_tortoise(c->stream, q.M, q.a, q.rstar_min, I.drs, q.n_rstar, I.off, I.x_int,
                               I.x_half);
        c->launches++;
        if (q.prec == TEUK_FP64 || q.prec == TEUK_FP64_DF) {  // the FP32 paths form theirs from 1D tables
            const teuk_status e = coef_tables(c, I);
            if (e != TEUK_OK) return fail(e);
        } else {
            TK_CCUDA(dmalloc(c, (void**)&I.rtab, sizeof(RTab2) * q.n_rstar, c->stream));
            TK_CCUDA(dmalloc(c, (void**)&I.thtab, sizeof(ThTab) * q.n_theta, c->stream));
            launch_tables_1d(c->stream, q.M, q.a, q.s, q.m, I.drs, I.dth, I.dt, q.n_rstar,
                             q.n_theta, I.x_int, I.x_half, I.rtab, I.thtab);
            c->launches++;
        }
        TK_CCUDA(cudaGetLastError());
        I.r_ext = 0;  // filled lazily from x at r*_ext when needed (adjoint loss)
    }
    if (refresh_partitions(c) != TEUK_OK) return fail(TEUK_ECUDA);
#undef TK_CCUDA
    *out = c;
    return TEUK_OK;
}

// ------------------------------------------------------------------ source

namespace {

void free_source(teuk_ctx* c, Instance& I) {
    void* ptrs[] = {I.P_win, I.amps, I.traj_buf};
    for (void* q : ptrs)
        if (q) dfree(c, q, c->stream);
    I.P_win = nullptr;
    I.amps = nullptr;
    I.traj_buf = nullptr;
    I.src_on = false;
    I.sd = SourceDev{};
}

// Gaussian widths of a source (absolute units, else cells; 0 cells means 4)
void source_widths(const Instance& I, const teuk_orbit* o, double* sr, double* stt) {
    *sr = o && o->sigma_rstar_abs > 0 ? o->sigma_rstar_abs
          : (o && o->sigma_rstar_cells > 0 ? o->sigma_rstar_cells : 4.0) * I.drs;
    *stt = o && o->sigma_theta_abs > 0 ? o->sigma_theta_abs
           : (o && o->sigma_theta_cells > 0 ? o->sigma_theta_cells : 4.0) * I.dth;
}

// Window of the nodes that can lie within 8 sigma of a centre in [rs_lo, rs_hi] x
// [th_lo, th_hi], with one node of margin (the kernels apply the exact cut)
void source_window(const Instance& I, double rs_lo, double rs_hi, double th_lo, double th_hi,
                   double sr, double stt, SourceDev& sd) {
    const teuk_params& q = I.p;
    const int nr = q.n_rstar, nth = q.n_theta;
    auto clampi = [](double v, int lo, int hi) {
        return v < lo ? lo : (v > hi ? hi : (int)v);
    };
    // (local indices: grid index - off)
    int ilo = clampi(std::floor((rs_lo - 8 * sr - q.rstar_min) / I.drs) - 1 - I.off, 0, nr - 1);
    int ihi = clampi(std::ceil((rs_hi + 8 * sr - q.rstar_min) / I.drs) + 1 - I.off, 0, nr - 1);
    int hlo = clampi(std::floor((rs_lo - 8 * sr - q.rstar_min) / I.drs - 0.5) - 1 - I.off, 0, nr - 2);
    int hhi = clampi(std::ceil((rs_hi + 8 * sr - q.rstar_min) / I.drs - 0.5) + 1 - I.off, 0, nr - 2);
    int jlo = clampi(std::floor((th_lo - 8 * stt) / I.dth - 0.5) - 1, 0, nth - 1);
    int jhi = clampi(std::ceil((th_hi + 8 * stt) / I.dth - 0.5) + 1, 0, nth - 1);
    sd.i_lo = ilo; sd.ni = ihi - ilo + 1;
    sd.h_lo = hlo; sd.nh = hhi - hlo + 1;
    sd.j_lo = jlo; sd.nj = jhi - jlo + 1;
}

}  // namespace

extern "C" teuk_status teuk_set_source(teuk_ctx* c, int instance, const teuk_orbit* orbit,
                                       const double* amps, int64_t n_amps) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    Instance& I = c->inst[instance];
    if (!orbit) TK_FAIL(c, TEUK_EINVAL, "orbit is NULL");
    if (n_amps < 0 || (n_amps > 0 && !amps)) TK_FAIL(c, TEUK_EINVAL, "bad amplitude array");
    const teuk_params& q = I.p;
    double r0 = orbit->r0;
    if (!(r0 > I.rp)) TK_FAIL(c, TEUK_EINVAL, "orbit radius r0=%g inside the horizon", r0);
    double rs0 = rstar_of_r(q.M, q.a, r0);
    if (!(rs0 > q.rstar_min && rs0 < q.rstar_max))
        TK_FAIL(c, TEUK_EINVAL, "orbit r*(r0)=%g outside the radial grid", rs0);
    double sr, stt;
    source_widths(I, orbit, &sr, &stt);
    // window of nodes that can be within 8 sigma (the kernel applies the exact cut)
    SourceDev sd{};
    source_window(I, rs0, rs0, 0.5 * kPi, 0.5 * kPi, sr, stt, sd);
    double Omega = std::sqrt(q.M) / (std::pow(r0, 1.5) + q.a * std::sqrt(q.M));
    double phi0 = q.a / (I.rp - I.rm) * std::log((r0 - I.rp) / (r0 - I.rm));
    double Delta0 = r0 * r0 - 2 * q.M * r0 + q.a * q.a;
    double dOmega = -std::sqrt(q.M) * 1.5 * std::sqrt(r0) /
                    ((std::pow(r0, 1.5) + q.a * std::sqrt(q.M)) * (std::pow(r0, 1.5) + q.a * std::sqrt(q.M)));
    sd.omega = q.m * Omega;
    sd.phase0 = q.m * phi0;
    sd.domega = q.m * dOmega;
    sd.dphase0 = q.m * q.a / Delta0;
    // (re)allocate window and amplitudes
    free_source(c, I);
    size_t nwi = (size_t)sd.nj * sd.ni, nwh = (size_t)sd.nj * sd.nh;
    // P, P_half, dP, dP_half (double2), then the step kernels' copies Q_int, Q_half
    const bool q16 = q.prec == TEUK_FP64 || q.prec == TEUK_FP64_DF;   // 16-byte profile entries
    const size_t qe = q16 ? 16 : sizeof(float2);
    sd.q_stride = q16 ? sd.nj : (sd.nj + 1) / 2 * 2;
    const size_t qi_bytes = qe * sd.q_stride * sd.ni, qh_bytes = qe * sd.q_stride * sd.nh;
    TK_CUDA(c, dmalloc(c, (void**)&I.P_win, sizeof(double2) * 2 * (nwi + nwh) + qi_bytes + qh_bytes,
                               c->stream));
    sd.P_int = I.P_win;
    sd.P_half = I.P_win + nwi;
    sd.dP_int = I.P_win + nwi + nwh;
    sd.dP_half = I.P_win + 2 * nwi + nwh;
    sd.Q_int = I.P_win + 2 * (nwi + nwh);
    sd.Q_half = (const char*)sd.Q_int + qi_bytes;
    if (n_amps > 0) {
        TK_CUDA(c, dmalloc(c, (void**)&I.amps, sizeof(double) * n_amps, c->stream));
        TK_CUDA(c, cudaMemcpyAsync(I.amps, amps, sizeof(double) * n_amps, cudaMemcpyHostToDevice,
                                   c->stream));
    }
    sd.amps = I.amps;
    sd.n_amps = n_amps;
    I.rs0 = rs0;
    I.sig_r = sr;
    I.sig_t = stt;
    I.drs0_dr0 = (r0 * r0 + q.a * q.a) / Delta0;
    launch_profile(c->stream, q.M, q.a, q.rstar_min, I.drs, I.off, I.dth, rs0, sr, stt, I.drs0_dr0,
                   I.x_int, I.x_half, sd, (int)q.prec);
    c->launches++;
    TK_CUDA(c, cudaGetLastError());
    I.sd = sd;
    I.orbit = *orbit;
    I.src_on = true;
    st = refresh_partition(c, I);
    if (st) return st;
    if (n_amps > 0) TK_CUDA(c, cudaStreamSynchronize(c->stream));  // host amps may be freed
    return TEUK_OK;
}

extern "C" teuk_status teuk_set_trajectory(teuk_ctx* c, int instance, const teuk_orbit* widths,
                                           const double* traj, int64_t n_samples) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    Instance& I = c->inst[instance];
    if (!traj || n_samples < 1) TK_FAIL(c, TEUK_EINVAL, "need a trajectory of at least one sample");
    if (n_samples > ((int64_t)1 << 31)) TK_FAIL(c, TEUK_EINVAL, "too many trajectory samples");
    const teuk_params& q = I.p;
    double r_lo = HUGE_VAL, r_hi = -HUGE_VAL, t_lo = HUGE_VAL, t_hi = -HUGE_VAL;
    for (int64_t k = 0; k < n_samples; ++k) {
        const double* smp = traj + 4 * k;
        if (!std::isfinite(smp[0]) || !std::isfinite(smp[1]) || !std::isfinite(smp[2]) ||
            !std::isfinite(smp[3]))
            TK_FAIL(c, TEUK_EINVAL, "trajectory sample %lld is not finite", (long long)k);
        if (!(smp[0] > I.rp))
            TK_FAIL(c, TEUK_EINVAL, "trajectory sample %lld: r_p=%g not outside the horizon",
                    (long long)k, smp[0]);
        if (!(smp[1] > 0.0 && smp[1] < kPi))
            TK_FAIL(c, TEUK_EINVAL, "trajectory sample %lld: theta_p=%g outside (0, pi)",
                    (long long)k, smp[1]);
        r_lo = std::fmin(r_lo, smp[0]);
        r_hi = std::fmax(r_hi, smp[0]);
        t_lo = std::fmin(t_lo, smp[1]);
        t_hi = std::fmax(t_hi, smp[1]);
    }
    const double rs_lo = rstar_of_r(q.M, q.a, r_lo), rs_hi = rstar_of_r(q.M, q.a, r_hi);
    if (!(rs_lo > q.rstar_min && rs_hi < q.rstar_max))
        TK_FAIL(c, TEUK_EINVAL, "the path leaves the radial grid (r* from %g to %g)", rs_lo, rs_hi);
    double sr, stt;
    source_widths(I, widths, &sr, &stt);
    SourceDev sd{};
    source_window(I, rs_lo, rs_hi, t_lo, t_hi, sr, stt, sd);
    sd.moving = 1;
    sd.n_traj = (n_samples + 1) / 2;
    // device memory: the profile Q (as for the circular orbit), then the samples, the
    // amplitudes and the radial and angular factor tables in the arithmetic type
    const bool q16 = q.prec == TEUK_FP64 || q.prec == TEUK_FP64_DF;
    const size_t qe = q16 ? 16 : sizeof(float2);
    sd.q_stride = q16 ? sd.nj : (sd.nj + 1) / 2 * 2;
    const size_t qi_bytes = qe * sd.q_stride * sd.ni, qh_bytes = qe * sd.q_stride * sd.nh;
    const size_t te = q16 ? 8 : 4;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_traj = up(sizeof(double) * 4 * (size_t)n_samples);
    const size_t b_amp = up(sizeof(double2) * 2 * (size_t)sd.n_traj);
    const size_t b_gr = up(te * (size_t)sd.n_traj * (sd.nh + sd.ni));
    const size_t b_gt = up(te * (size_t)sd.n_traj * 2 * sd.nj);
    free_source(c, I);
    TK_CUDA(c, dmalloc(c, (void**)&I.P_win, qi_bytes + qh_bytes, c->stream));
    TK_CUDA(c, dmalloc(c, &I.traj_buf, b_traj + b_amp + b_gr + b_gt, c->stream));
    sd.Q_int = I.P_win;
    sd.Q_half = (const char*)sd.Q_int + qi_bytes;
    char* tb = (char*)I.traj_buf;
    const double* d_traj = (const double*)tb;
    sd.amp = (const double2*)(tb + b_traj);
    sd.gr = tb + b_traj + b_amp;
    sd.gt = tb + b_traj + b_amp + b_gr;
    TK_CUDA(c, cudaMemcpyAsync((void*)d_traj, traj, sizeof(double) * 4 * (size_t)n_samples,
                               cudaMemcpyHostToDevice, c->stream));
    launch_trajectory(c->stream, q.M, q.a, q.m, q.rstar_min, I.drs, I.off, I.dth, sr, stt, I.x_int, I.x_half,
                      d_traj, n_samples, sd, (int)q.prec);
    c->launches += 2;
    TK_CUDA(c, cudaGetLastError());
    I.sd = sd;
    I.orbit = widths ? *widths : teuk_orbit{};
    I.sig_r = sr;
    I.sig_t = stt;
    I.src_on = true;
    st = refresh_partition(c, I);
    if (st) return st;
    TK_CUDA(c, cudaStreamSynchronize(c->stream));  // the host samples may be freed
    return TEUK_OK;
}

// ------------------------------------------------------------------ state

extern "C" teuk_status teuk_set_state(teuk_ctx* c, int instance, const double* host_u,
                                      int64_t step0) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    if (!host_u || step0 < 0) TK_FAIL(c, TEUK_EINVAL, "host_u is NULL or step0 < 0");
    Instance& I = c->inst[instance];
    size_t bytes = sizeof(double) * 4 * (size_t)I.p.n_rstar * I.p.n_theta;
    if (!I.stage) TK_CUDA(c, dmalloc(c, (void**)&I.stage, bytes, c->stream));
    TK_CUDA(c, cudaMemcpyAsync(I.stage, host_u, bytes, cudaMemcpyHostToDevice, c->stream));
    launch_import_state(c->stream, dev_of(c, I), I.cur, I.stage);
    c->launches++;
    TK_CUDA(c, cudaGetLastError());
    TK_CUDA(c, cudaStreamSynchronize(c->stream));  // the host buffer may go away after return
    I.step = step0;
    I.wave_lo = I.wave_hi = step0;
    return TEUK_OK;
}

extern "C" teuk_status teuk_get_state(teuk_ctx* c, int instance, double* host_u) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    if (!host_u) TK_FAIL(c, TEUK_EINVAL, "host_u is NULL");
    Instance& I = c->inst[instance];
    size_t bytes = sizeof(double) * 4 * (size_t)I.p.n_rstar * I.p.n_theta;
    if (!I.stage) TK_CUDA(c, dmalloc(c, (void**)&I.stage, bytes, c->stream));
    launch_export_state(c->stream, dev_of(c, I), I.cur, I.stage);
    c->launches++;
    TK_CUDA(c, cudaGetLastError());
    TK_CUDA(c, cudaMemcpyAsync(host_u, I.stage, bytes, cudaMemcpyDeviceToHost, c->stream));
    TK_CUDA(c, cudaStreamSynchronize(c->stream));
    return TEUK_OK;
}

// ------------------------------------------------------------------ checkpoint / resume
// File: 8-byte magic, then the fields below (host byte order), then the planes of the
// current level, each plane_bytes long, in the library's own layout.

namespace {

constexpr char kStateMagic[8] = {'T', 'E', 'U', 'K', 'S', 'T', '0', '1'};

struct StateFileHeader {
    int32_t s, m, n_rstar, n_theta, dt_rule, prec, slab_col0, slab_ncols;
    double M, a, rstar_min, rstar_max, courant, dt, rstar_ext;
    int64_t step;
    uint64_t plane_bytes;
    int32_t nplanes, pad;
};

StateFileHeader header_of(const Instance& I) {
    const teuk_params& q = I.p;
    StateFileHeader h{};
    h.s = q.s; h.m = q.m; h.n_rstar = q.n_rstar; h.n_theta = q.n_theta; h.dt_rule = q.dt_rule;
    h.prec = q.prec; h.slab_col0 = q.slab_col0; h.slab_ncols = q.slab_ncols;
    h.M = q.M; h.a = q.a; h.rstar_min = q.rstar_min; h.rstar_max = q.rstar_max;
    h.courant = q.courant; h.dt = q.dt; h.rstar_ext = q.rstar_ext;
    h.step = I.step;
    h.plane_bytes = I.plane_bytes;
    h.nplanes = I.p.prec == TEUK_FP32 ? 1 : 2;
    return h;
}

// the saved problem is this instance's: every parameter but the waveform capacity
bool same_problem(const StateFileHeader& a, const StateFileHeader& b) {
    return a.s == b.s && a.m == b.m && a.n_rstar == b.n_rstar && a.n_theta == b.n_theta &&
           a.dt_rule == b.dt_rule && a.prec == b.prec && a.slab_col0 == b.slab_col0 &&
           a.slab_ncols == b.slab_ncols && a.M == b.M && a.a == b.a && a.rstar_min == b.rstar_min &&
           a.rstar_max == b.rstar_max && a.courant == b.courant && a.dt == b.dt &&
           a.rstar_ext == b.rstar_ext && a.plane_bytes == b.plane_bytes && a.nplanes == b.nplanes;
}

}  // namespace

extern "C" teuk_status teuk_save_state(teuk_ctx* c, int instance, const char* path) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    if (!path) TK_FAIL(c, TEUK_EINVAL, "path is NULL");
    Instance& I = c->inst[instance];
    const StateFileHeader h = header_of(I);
    std::vector<char> buf((size_t)h.nplanes * I.plane_bytes);
    for (int k = 0; k < h.nplanes; ++k)
        TK_CUDA(c, cudaMemcpyAsync(buf.data() + (size_t)k * I.plane_bytes, I.state[I.cur][k], I.plane_bytes,
                                   cudaMemcpyDeviceToHost, c->stream));
    TK_CUDA(c, cudaStreamSynchronize(c->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) TK_FAIL(c, TEUK_EINVAL, "cannot open %s for writing", path);
    const bool ok = std::fwrite(kStateMagic, 1, 8, f) == 8 && std::fwrite(&h, sizeof h, 1, f) == 1 &&
                    std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) TK_FAIL(c, TEUK_EINVAL, "writing %s failed", path);
    return TEUK_OK;
}

extern "C" teuk_status teuk_load_state(teuk_ctx* c, int instance, const char* path) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    if (!path) TK_FAIL(c, TEUK_EINVAL, "path is NULL");
    Instance& I = c->inst[instance];
    const StateFileHeader want = header_of(I);
    FILE* f = std::fopen(path, "rb");
    if (!f) TK_FAIL(c, TEUK_EINVAL, "cannot open %s", path);
    char magic[8] = {};
    StateFileHeader h{};
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kStateMagic, 8) == 0 &&
              std::fread(&h, sizeof h, 1, f) == 1;
    if (!ok || !same_problem(h, want) || h.step < 0) {
        std::fclose(f);
        TK_FAIL(c, TEUK_EINVAL, "%s is not a saved state of this instance's problem", path);
    }
    std::vector<char> buf((size_t)h.nplanes * I.plane_bytes);
    ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) TK_FAIL(c, TEUK_EINVAL, "%s is truncated", path);
    for (int k = 0; k < h.nplanes; ++k)
        TK_CUDA(c, cudaMemcpyAsync(I.state[I.cur][k], buf.data() + (size_t)k * I.plane_bytes, I.plane_bytes,
                                   cudaMemcpyHostToDevice, c->stream));
    TK_CUDA(c, cudaStreamSynchronize(c->stream));   // the host buffer goes away on return
    I.step = h.step;
    I.wave_lo = I.wave_hi = h.step;
    return TEUK_OK;
}

// ------------------------------------------------------------------ step

namespace {

void invalidate_graph(teuk_ctx* c) {
    Batch& B = c->batch;
    if (B.exec) cudaGraphExecDestroy(B.exec);
    if (B.graph) cudaGraphDestroy(B.graph);
    B.exec = nullptr;
    B.graph = nullptr;
}

void enqueue_batched(teuk_ctx* c, cudaStream_t st) {
    Batch& B = c->batch;
    cudaMemsetAsync(B.d_abort, 0, sizeof(int), st);
    for (BatchClass& K : B.cls) {
        cudaMemsetAsync(K.d_counter, 0, sizeof(unsigned long long), st);
        cudaMemsetAsync(K.d_flags, 0, sizeof(int) * K.items, st);
    }
    for (BatchClass& K : B.cls) launch_batched_step(st, c->prec, K.bd, K.grid, K.pitch, K.moving);
    for (BatchClass& K : B.cls) launch_batched_extract(st, c->prec, K.bd, K.max_nth);
}

// All instances advance n steps: one persistent launch per block-size class, captured
// once in a CUDA graph and replayed (the per-call descriptors are uploaded first).
teuk_status batched_step(teuk_ctx* c, int64_t n) {
    Batch& B = c->batch;
    const int ni = (int)c->inst.size();
    if (B.cls.empty()) {
        for (int k = 0; k < ni; ++k) {
            int pitch = c->inst[k].pitch;
            BatchClass* K = nullptr;
            for (BatchClass& q : B.cls)
                if (q.pitch == pitch) K = &q;
            if (!K) {
                B.cls.emplace_back();
                K = &B.cls.back();
                K->pitch = pitch;
            }
            K->members.push_back(k);
        }
    }
    // per-class descriptor blocks:
    // InstDev[m] | item_base[m+1] | base_step[m] | n_steps | strip[m] | nstrip[m] | base_bin[m]
    std::vector<char> blob;
    bool changed = false;
    for (BatchClass& K : B.cls) {
        const int m = (int)K.members.size();
        size_t off = (blob.size() + 255) / 256 * 256;
        K.off = off;
        size_t o_inst = off, o_ib = o_inst + sizeof(InstDev) * m;
        size_t o_bs = o_ib + sizeof(int64_t) * (m + 1), o_n = o_bs + sizeof(int64_t) * m;
        size_t o_st = o_n + sizeof(int64_t), o_ns = o_st + sizeof(int) * m;
        size_t o_bb = o_ns + sizeof(int) * m, end = o_bb + sizeof(int) * m;
        blob.resize(end);
        std::vector<int64_t> ib(m + 1, 0), bs(m);
        std::vector<int> strip(m), nstrip(m), bb(m);
        std::vector<InstDev> idev(m);
        int max_nth = 0;
        bool moving = false;
        for (int q = 0; q < m; ++q) {
            Instance& I = c->inst[K.members[q]];
            strip[q] = eff_strip(c, I);
            nstrip[q] = (I.p.n_rstar - 2 + strip[q] - 1) / strip[q];
            ib[q + 1] = ib[q] + nstrip[q];
            bs[q] = I.step;
            bb[q] = I.cur;
            idev[q] = dev_of(c, I);
            max_nth = std::max(max_nth, I.p.n_theta);
            moving = moving || (I.src_on && I.sd.moving);
        }
        std::memcpy(blob.data() + o_inst, idev.data(), sizeof(InstDev) * m);
        std::memcpy(blob.data() + o_ib, ib.data(), sizeof(int64_t) * (m + 1));
        std::memcpy(blob.data() + o_bs, bs.data(), sizeof(int64_t) * m);
        std::memcpy(blob.data() + o_n, &n, sizeof(int64_t));
        std::memcpy(blob.data() + o_st, strip.data(), sizeof(int) * m);
        std::memcpy(blob.data() + o_ns, nstrip.data(), sizeof(int) * m);
        std::memcpy(blob.data() + o_bb, bb.data(), sizeof(int) * m);
        if (ib[m] != K.items || max_nth != K.max_nth || moving != K.moving) changed = true;
        K.moving = moving;
        K.items = ib[m];
        K.max_nth = max_nth;
        K.bd.n_inst = m;
        K.bd.items_per_step = K.items;
        K.bd.status = c->status;
        if (K.bd.spin_limit != c->spin_limit || K.bd.skip_release_item != c->inject_skip_item)
            changed = true;
        K.bd.spin_limit = c->spin_limit;          // default ~1.3 s of 64 ns sleeps per wait
        K.bd.skip_release_item = c->inject_skip_item;
        // pointers into the device blob (set below once it exists)
        K.bd.inst = (const InstDev*)(uintptr_t)o_inst;
        K.bd.item_base = (const int64_t*)(uintptr_t)o_ib;
        K.bd.base_step = (const int64_t*)(uintptr_t)o_bs;
        K.bd.n_steps = (const int64_t*)(uintptr_t)o_n;
        K.bd.strip = (const int*)(uintptr_t)o_st;
        K.bd.nstrip = (const int*)(uintptr_t)o_ns;
        K.bd.base_bin = (const int*)(uintptr_t)o_bb;
    }
    if (!B.alloc) {
        TK_CUDA(c, dmalloc(c, (void**)&B.d_blob, blob.size(), c->stream));
        TK_CUDA(c, dmalloc(c, (void**)&B.d_abort, sizeof(int), c->stream));
        B.blob_bytes = blob.size();
        for (BatchClass& K : B.cls) {
            TK_CUDA(c, dmalloc(c, (void**)&K.d_counter, sizeof(unsigned long long), c->stream));
            K.grid = batched_grid(c->prec, K.pitch);
        }
        B.alloc = true;
        changed = true;
    }
    for (BatchClass& K : B.cls) {
        if (K.items > K.flags_cap) {
            if (K.d_flags) dfree(c, K.d_flags, c->stream);
            TK_CUDA(c, dmalloc(c, (void**)&K.d_flags, sizeof(int) * K.items, c->stream));
            K.flags_cap = K.items;
            changed = true;
        }
        char* base = B.d_blob;
        K.bd.inst = (const InstDev*)(base + (uintptr_t)K.bd.inst);
        K.bd.item_base = (const int64_t*)(base + (uintptr_t)K.bd.item_base);
        K.bd.base_step = (const int64_t*)(base + (uintptr_t)K.bd.base_step);
        K.bd.n_steps = (const int64_t*)(base + (uintptr_t)K.bd.n_steps);
        K.bd.strip = (const int*)(base + (uintptr_t)K.bd.strip);
        K.bd.nstrip = (const int*)(base + (uintptr_t)K.bd.nstrip);
        K.bd.base_bin = (const int*)(base + (uintptr_t)K.bd.base_bin);
        K.bd.counter = K.d_counter;
        K.bd.flags = K.d_flags;
        K.bd.abort = B.d_abort;
    }
    if (changed) invalidate_graph(c);
    // pageable source: the call returns once the host bytes are staged
    TK_CUDA(c, cudaMemcpyAsync(B.d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice,
                               c->stream));
    cudaStreamCaptureStatus ucs = cudaStreamCaptureStatusNone;
    const bool user_capturing = cudaStreamIsCapturing(c->stream, &ucs) != cudaSuccess ||
                                ucs != cudaStreamCaptureStatusNone;
    cudaGetLastError();
    cudaStream_t cs = user_capturing ? nullptr : capture_stream(c);
    if (!B.exec && !B.graph_failed && cs) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            enqueue_batched(c, cs);
            if (cudaStreamEndCapture(cs, &g) == cudaSuccess && g &&
                cudaGraphInstantiate(&B.exec, g, 0) == cudaSuccess) {
                B.graph = g;
            } else {
                if (g) cudaGraphDestroy(g);
                B.exec = nullptr;
                B.graph_failed = true;
            }
        } else {
            B.graph_failed = true;
        }
        cudaGetLastError();  // a refused capture is not an error here
    }
    if (B.exec && !user_capturing) {
        TK_CUDA(c, cudaGraphLaunch(B.exec, c->stream));
    } else {
        enqueue_batched(c, c->stream);
    }
    c->launches += 2 * (int64_t)B.cls.size();
    for (Instance& I : c->inst) {
        int64_t s0 = I.step;
        I.step += n;
        I.cur = (int)((I.cur + n) & 1);
        if (I.wave_hi != s0 + 1 || I.wave_lo == I.wave_hi) I.wave_lo = s0;
        I.wave_hi = I.step + 1;
        if (I.wave_hi - I.wave_lo > I.wave_cap) I.wave_lo = I.wave_hi - I.wave_cap;
    }
    TK_CUDA(c, cudaGetLastError());
    return TEUK_OK;
}

}  // namespace

namespace {

// Plan the resident launch of instance I with halo h, aiming at bps blocks per SM, and
// (re)allocate its exchange slots and flags; h = 0 turns resident launches off.
teuk_status set_resident(teuk_ctx* c, Instance& I, int h, int bps, bool blocked = false) {
    if (h == 0) {
        I.res_h = 0;
        I.res_blocked = false;
        return TEUK_OK;
    }
    ResidentPlan plan;
    if (!resident_plan(I.p.prec, I.p.n_rstar, I.pitch, h, bps, &plan))
        TK_FAIL(c, TEUK_EINVAL,
                "the grid does not fit the resident kernel with halo %d and %d blocks per SM (every "
                "block must own >= %d columns, hold its columns in shared memory and be resident "
                "at once)", h, bps, h);
    const int planes = I.p.prec == TEUK_FP32 ? 1 : 2;
    const size_t xg_bytes = (size_t)planes * 2 * plan.nb * 2 * h * I.pitch * 16;
    if (I.res_xg) dfree(c, I.res_xg, c->stream);
    if (I.res_flags) dfree(c, I.res_flags, c->stream);
    I.res_xg = nullptr;
    I.res_flags = nullptr;
    I.res_h = 0;
    TK_CUDA(c, dmalloc(c, (void**)&I.res_xg, xg_bytes, c->stream));
    TK_CUDA(c, dmalloc(c, (void**)&I.res_flags, sizeof(int) * kResFlagStride * (plan.nb + 1), c->stream));
    I.res_plan = plan;
    I.res_h = h;
    I.res_bps = bps;
    I.res_blocked = blocked;
    return TEUK_OK;
}

// n steps of a single instance in one cooperative launch of the resident kernel, then the
// record of the final level (the kernel records the levels it starts each step from).
teuk_status resident_step(teuk_ctx* c, Instance& I, int64_t n) {
    ResidentArgs a{};
    a.d = dev_of(c, I);
    a.step0 = I.step;
    a.bin = I.cur;
    a.obin = (int)((I.cur + n) & 1);
    a.n = n;
    a.h = I.res_plan.h;
    a.nb = I.res_plan.nb;
    a.xg = I.res_xg;
    a.flags = I.res_flags;
    a.abort = I.res_flags + (size_t)kResFlagStride * I.res_plan.nb;
    a.skip_publish = (int)c->inject_skip_item;
    a.no_wait = 0;
    TK_CUDA(c, cudaMemsetAsync(I.res_flags, 0, sizeof(int) * kResFlagStride * (I.res_plan.nb + 1), c->stream));
    TK_CUDA(c, launch_resident(c->stream, a, I.res_plan));
    c->launches++;
    I.step += n;
    I.cur = a.obin;
    do_extract(c, I);
    return TEUK_OK;
}

// n steps of a single instance in blocked launches: each takes at most h steps of the grid
// held in shared memory, reading its halo columns from the previous launch's output, and
// writes the other buffer (the launch boundary is the synchronisation: no flag waits);
// then the record of the final level.
teuk_status blocked_step(teuk_ctx* c, Instance& I, int64_t n) {
    for (int64_t done = 0; done < n;) {
        const int64_t k = std::min<int64_t>(n - done, I.res_plan.h);
        ResidentArgs a{};
        a.d = dev_of(c, I);
        a.step0 = I.step;
        a.bin = I.cur;
        a.obin = 1 - I.cur;
        a.n = k;
        a.h = I.res_plan.h;
        a.nb = I.res_plan.nb;
        a.xg = I.res_xg;
        a.flags = I.res_flags;
        a.abort = I.res_flags + (size_t)kResFlagStride * I.res_plan.nb;
        a.skip_publish = -1;
        a.no_wait = 1;
        TK_CUDA(c, launch_resident(c->stream, a, I.res_plan, false));
        c->launches++;
        I.step += k;
        I.cur = a.obin;
        done += k;
    }
    do_extract(c, I);
    return TEUK_OK;
}

}  // namespace

extern "C" teuk_status teuk_set_allocator(teuk_alloc_fn alloc, teuk_free_fn free_fn, void* user) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        g_create_err = "teuk_set_allocator: give both functions, or neither";
        return TEUK_EINVAL;
    }
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.user = alloc ? user : nullptr;
    return TEUK_OK;
}

extern "C" teuk_status teuk_set_resident_shape(teuk_ctx* c, int halo, int blocks_per_sm) {
    if (!c) return TEUK_EINVAL;
    if (halo < 0) TK_FAIL(c, TEUK_EINVAL, "halo must be >= 0");
    if (blocks_per_sm < 1) TK_FAIL(c, TEUK_EINVAL, "blocks_per_sm must be >= 1");
    if (c->inst.size() != 1) TK_FAIL(c, TEUK_EINVAL, "resident launches serve single-instance contexts");
    if (halo > 0 && c->inst[0].slab)
        TK_FAIL(c, TEUK_EINVAL, "a slab takes its halo columns between steps: no resident launches");
    return set_resident(c, c->inst[0], halo, blocks_per_sm);
}

extern "C" teuk_status teuk_set_resident(teuk_ctx* c, int halo) {
    return teuk_set_resident_shape(c, halo, 1);
}

extern "C" teuk_status teuk_set_blocked(teuk_ctx* c, int steps, int blocks_per_sm) {
    if (!c) return TEUK_EINVAL;
    if (steps < 0) TK_FAIL(c, TEUK_EINVAL, "steps must be >= 0");
    if (blocks_per_sm < 1) TK_FAIL(c, TEUK_EINVAL, "blocks_per_sm must be >= 1");
    if (c->inst.size() != 1) TK_FAIL(c, TEUK_EINVAL, "blocked launches serve single-instance contexts");
    if (steps > 0 && c->inst[0].slab)
        TK_FAIL(c, TEUK_EINVAL, "a slab takes its halo columns between steps: no blocked launches");
    return set_resident(c, c->inst[0], steps, blocks_per_sm, true);
}

extern "C" teuk_status teuk_step_n(teuk_ctx* c, int64_t n) {
    if (!c) return TEUK_EINVAL;
    if (n < 0) TK_FAIL(c, TEUK_EINVAL, "n < 0");
    if (n == 0) return TEUK_OK;
    if (c->inst.size() > 1 || c->steps_per_launch == 0) return batched_step(c, n);
    Instance& I0 = c->inst[0];
    if (I0.res_h > 0 && !(I0.src_on && I0.sd.moving)) {   // a moving particle: per-step launches
        const int64_t s0 = I0.step;
        teuk_status st = I0.res_blocked ? blocked_step(c, I0, n) : resident_step(c, I0, n);
        if (st) return st;
        if (I0.wave_hi != s0 + 1 || I0.wave_lo == I0.wave_hi) I0.wave_lo = s0;
        I0.wave_hi = I0.step + 1;
        if (I0.wave_hi - I0.wave_lo > I0.wave_cap) I0.wave_lo = I0.wave_hi - I0.wave_cap;
        TK_CUDA(c, cudaGetLastError());
        return TEUK_OK;
    }
    for (Instance& I : c->inst) {
        int strip = eff_strip(c, I);
        int64_t s0 = I.step;
        int64_t k = 0;
        // whole graphs of kStepGraph steps, then the rest one launch at a time
        cudaGraphExec_t e = n >= kStepGraph ? step_graph(c, I, strip) : nullptr;
        if (e) {
            if (I.graph_base != I.step) {   // the base the graph's steps are offsets from
                I.h_step = I.step;
                TK_CUDA(c, cudaMemcpyAsync(I.d_step, &I.h_step, sizeof(int64_t), cudaMemcpyHostToDevice,
                                           c->stream));
                I.graph_base = I.step;
            }
            for (; k + kStepGraph <= n; k += kStepGraph) {
                TK_CUDA(c, cudaGraphLaunch(e, c->stream));
                c->launches += kStepGraph + 1;
                I.step += kStepGraph;
                I.graph_base += kStepGraph;   // advanced by the graph's last node
            }
        }
        for (; k < n; ++k) do_step(c, I, strip);
        do_extract(c, I);
        if (I.wave_hi != s0 + 1 || I.wave_lo == I.wave_hi) I.wave_lo = s0;
        I.wave_hi = I.step + 1;
        if (I.wave_hi - I.wave_lo > I.wave_cap) I.wave_lo = I.wave_hi - I.wave_cap;
    }
    TK_CUDA(c, cudaGetLastError());
    return TEUK_OK;
}

extern "C" teuk_status teuk_extract(teuk_ctx* c, int instance, double* out, double* out_scalar,
                                    int64_t cap_steps, int64_t* n_written, int64_t* first_step) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    if (cap_steps < 0 || (cap_steps > 0 && !out)) TK_FAIL(c, TEUK_EINVAL, "bad output buffer");
    Instance& I = c->inst[instance];
    if (!I.ext_here)
        TK_FAIL(c, TEUK_EINVAL, "instance %d is a slab that does not hold the extraction radius", instance);
    int64_t held = I.wave_hi - I.wave_lo;
    int64_t k = std::min(cap_steps, held);
    int64_t lvl0 = I.wave_hi - k;
    int nth = I.p.n_theta;
    size_t rec = sizeof(double2) * nth;
    // copy in at most two segments of the ring
    int64_t done = 0;
    while (done < k) {
        int64_t slot = (lvl0 + done) % I.wave_cap;
        int64_t run = std::min(k - done, I.wave_cap - slot);
        TK_CUDA(c, cudaMemcpyAsync(out + done * 2 * nth, I.wave + slot * nth, rec * run,
                                   cudaMemcpyDeviceToHost, c->stream));
        done += run;
    }
    if (out_scalar && k > 0) {
        if (k > c->sum_cap) {
            if (c->sum_buf) dfree(c, c->sum_buf, c->stream);
            c->sum_buf = nullptr;
            c->sum_cap = 0;
            TK_CUDA(c, dmalloc(c, (void**)&c->sum_buf, sizeof(double2) * k, c->stream));
            c->sum_cap = k;
        }
        launch_wave_sum(c->stream, I.wave, I.wave_cap, nth, I.dth, lvl0, k, c->sum_buf);
        c->launches++;
        TK_CUDA(c, cudaGetLastError());
        TK_CUDA(c, cudaMemcpyAsync(out_scalar, c->sum_buf, sizeof(double2) * k, cudaMemcpyDeviceToHost,
                                   c->stream));
    }
    TK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (n_written) *n_written = k;
    if (first_step) *first_step = lvl0;
    return TEUK_OK;
}

namespace {
double r_of_rstar_host(double M, double a, double target);
}  // namespace

// The instances as modes of one problem (the same s, M, a, n_theta, time step and
// extraction radius), each holding the records first .. first + n_records - 1.
static teuk_status modes_of_problem(teuk_ctx* c, int64_t first, int64_t n_records,
                                    std::vector<ModeRing>& modes) {
    const Instance& I0 = c->inst[0];
    const int nth = I0.p.n_theta;
    modes.resize(c->inst.size());
    for (size_t i = 0; i < c->inst.size(); ++i) {
        const Instance& I = c->inst[i];
        if (I.p.s != I0.p.s || I.p.M != I0.p.M || I.p.a != I0.p.a || I.p.n_theta != nth ||
            I.dt != I0.dt || I.p.rstar_ext != I0.p.rstar_ext)
            TK_FAIL(c, TEUK_EINVAL,
                    "instance %d is not a mode of instance 0's problem (s, M, a, n_theta, time step "
                    "and extraction radius must agree; set dt to share the step)", (int)i);
        if (!I.ext_here)
            TK_FAIL(c, TEUK_EINVAL, "instance %d is a slab that does not hold the extraction radius", (int)i);
        if (first < I.wave_lo || first + n_records > I.wave_hi)
            TK_FAIL(c, TEUK_EINVAL, "instance %d holds records [%lld, %lld), not [%lld, %lld)", (int)i,
                    (long long)I.wave_lo, (long long)I.wave_hi, (long long)first,
                    (long long)(first + n_records));
        modes[i] = ModeRing{I.wave, I.wave_cap, I.p.m, 0};
    }
    return TEUK_OK;
}

extern "C" teuk_status teuk_mode_sum(teuk_ctx* c, const double* phi, int n_phi, int64_t first,
                                     int64_t n_records, double* out) {
    if (!c) return TEUK_EINVAL;
    if (n_phi < 1 || !phi || n_records < 0 || (n_records > 0 && !out))
        TK_FAIL(c, TEUK_EINVAL, "need n_phi >= 1, phi, n_records >= 0 and an output buffer");
    const Instance& I0 = c->inst[0];
    const int nth = I0.p.n_theta;
    std::vector<ModeRing> modes;
    const teuk_status ms = modes_of_problem(c, first, n_records, modes);
    if (ms != TEUK_OK) return ms;
    if (n_records == 0) return TEUK_OK;
    // Eq. (3): phi~ = phi + a/(r_+ - r_-) ln((r - r_+)/(r - r_-)) at the extraction radius;
    // Eq. (4): Psi = e^{i m phi~} r^3 Phi
    const double r_ext = r_of_rstar_host(I0.p.M, I0.p.a, I0.p.rstar_ext);
    const double shift = I0.p.a / (I0.rp - I0.rm) * std::log((r_ext - I0.rp) / (r_ext - I0.rm));
    const size_t n_out = (size_t)n_records * nth * n_phi;
    char* buf = nullptr;
    const size_t b_modes = (sizeof(ModeRing) * modes.size() + 255) / 256 * 256;
    const size_t b_phi = (sizeof(double) * n_phi + 255) / 256 * 256;
    TK_CUDA(c, dmalloc(c, (void**)&buf, b_modes + b_phi + sizeof(double2) * n_out, c->stream));
    ModeRing* d_modes = (ModeRing*)buf;
    double* d_phi = (double*)(buf + b_modes);
    double2* d_out = (double2*)(buf + b_modes + b_phi);
    cudaMemcpyAsync(d_modes, modes.data(), sizeof(ModeRing) * modes.size(), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_phi, phi, sizeof(double) * n_phi, cudaMemcpyHostToDevice, c->stream);
    launch_mode_sum(c->stream, d_modes, (int)modes.size(), nth, d_phi, n_phi, first, n_records,
                    r_ext * r_ext * r_ext, shift, d_out);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d_out, sizeof(double2) * n_out, cudaMemcpyDeviceToHost, c->stream);
    dfree(c, buf, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) TK_FAIL(c, TEUK_ECUDA, "mode sum: %s", cudaGetErrorString(e));
    return TEUK_OK;
}

extern "C" teuk_status teuk_radiated_flux(teuk_ctx* c, int64_t first, int64_t n_records, double* out) {
    if (!c) return TEUK_EINVAL;
    if (n_records < 0 || (n_records > 0 && !out))
        TK_FAIL(c, TEUK_EINVAL, "need n_records >= 0 and an output buffer");
    std::vector<ModeRing> modes;
    const teuk_status ms = modes_of_problem(c, first, n_records, modes);
    if (ms != TEUK_OK) return ms;
    const int K = (int)modes.size();
    std::vector<int> partner(K, -1);
    for (int i = 0; i < K; ++i)
        for (int k = 0; k < K; ++k) {
            if (k != i && modes[k].m == modes[i].m)
                TK_FAIL(c, TEUK_EINVAL, "instances %d and %d are the same mode m = %d", i, k, modes[i].m);
            if (modes[k].m == modes[i].m + 1) partner[i] = k;
        }
    if (n_records == 0) return TEUK_OK;
    const Instance& I0 = c->inst[0];
    const int nth = I0.p.n_theta;
    const int64_t E = (int64_t)K * nth;
    const double r_ext = r_of_rstar_host(I0.p.M, I0.p.a, I0.p.rstar_ext);
    const double shift = I0.p.a / (I0.rp - I0.rm) * std::log((r_ext - I0.rp) / (r_ext - I0.rm));
    // rows in groups of RB: a block of K RB <= 256 threads, whole warps
    if (K > 256) TK_FAIL(c, TEUK_EINVAL, "radiated flux: at most 256 modes (got %d)", K);
    const int RB = std::max(1, std::min(256 / K, nth));
    const int n_rg = (nth + RB - 1) / RB;
    // chunks of the time scans: about 155 648 (152 SMs x 1024) integrating threads, their
    // starts and totals in at most 128 MB, at most 65535 chunks (the grid's y extent)
    int64_t n_chunks = (152 * 1024 + E - 1) / E;
    if (n_chunks * E * 64 > ((int64_t)128 << 20)) n_chunks = std::max<int64_t>(1, ((int64_t)128 << 20) / (E * 64));
    n_chunks = std::min<int64_t>(std::min<int64_t>(n_chunks, n_records), 65535);
    const int64_t Lc = (n_records + n_chunks - 1) / n_chunks;
    n_chunks = (n_records + Lc - 1) / Lc;
    if (Lc > INT32_MAX)
        TK_FAIL(c, TEUK_EINVAL, "radiated flux: %lld records are too many", (long long)n_records);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_modes = al(sizeof(ModeRing) * K), b_part = al(sizeof(int) * K);
    const size_t b_chunk = al(sizeof(double2) * (size_t)n_chunks * E);
    const size_t b_g = al(sizeof(FluxWeights) * (size_t)E), b_gp = al(sizeof(double2) * (size_t)E);
    const size_t b_sums = al(sizeof(double) * 5 * (size_t)n_rg * (size_t)n_records);
    const size_t b_out = sizeof(double) * 10 * (size_t)n_records;
    char* buf = nullptr;
    TK_CUDA(c, dmalloc(c, (void**)&buf, b_modes + b_part + 4 * b_chunk + b_g + b_gp + b_sums + b_out,
                       c->stream));
    char* q = buf;
    auto take = [&](size_t b) { char* r = q; q += b; return r; };
    ModeRing* d_modes = (ModeRing*)take(b_modes);
    int* d_part = (int*)take(b_part);
    FluxScratch fs;
    fs.totN = (double2*)take(b_chunk);
    fs.totH = (double2*)take(b_chunk);
    fs.stN = (double2*)take(b_chunk);
    fs.stH = (double2*)take(b_chunk);
    fs.g = (FluxWeights*)take(b_g);
    fs.gp = (double2*)take(b_gp);
    fs.partner = d_part;
    fs.part = (double*)take(b_sums);
    fs.out = (double*)take(b_out);
    cudaMemcpyAsync(d_modes, modes.data(), sizeof(ModeRing) * K, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_part, partner.data(), sizeof(int) * K, cudaMemcpyHostToDevice, c->stream);
    const FluxDev f{d_modes, K, nth, first, n_records, (int)Lc, (int)n_chunks, RB, n_rg,
                    I0.dt, r_ext, I0.p.a, shift};
    c->launches += launch_radiated_flux(c->stream, f, fs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, fs.out, b_out, cudaMemcpyDeviceToHost, c->stream);
    dfree(c, buf, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) TK_FAIL(c, TEUK_ECUDA, "radiated flux: %s", cudaGetErrorString(e));
    return TEUK_OK;
}

extern "C" int teuk_checked_build(void) {
#ifdef TEUK_CHECK
    return 1;
#else
    return 0;
#endif
}

extern "C" teuk_status teuk_check_selftest(teuk_ctx* c) {
    if (!c) return TEUK_EINVAL;
    if (!teuk_checked_build()) TK_FAIL(c, TEUK_EINVAL, "not a checked build (libteuk_check.so)");
    launch_check_selftest(c->stream, dev_of(c, c->inst[0]));
    c->launches++;
    TK_CUDA(c, cudaGetLastError());
    return TEUK_OK;
}

extern "C" teuk_status teuk_sync(teuk_ctx* c) {
    if (!c) return TEUK_EINVAL;
    for (Instance& I : c->inst) {
        launch_scan_finite(c->stream, dev_of(c, I), I.cur);
        c->launches++;
    }
    TK_CUDA(c, cudaGetLastError());
    unsigned h = 0;
    TK_CUDA(c, cudaMemcpyAsync(&h, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    TK_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));  // reported once
    TK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h & ST_TIMEOUT) TK_FAIL(c, TEUK_ETIMEOUT, "a bounded device wait gave up");
    if (h & ST_NONFINITE) TK_FAIL(c, TEUK_EUNSTABLE, "non-finite values in the state or waveform");
    if (h & ST_BOUNDS) TK_FAIL(c, TEUK_EBOUNDS, "a device-side index check failed (checked build)");
    return TEUK_OK;
}

extern "C" teuk_status teuk_get_time(const teuk_ctx* c, int instance, int64_t* step, double* dt) {
    if (!c || instance < 0 || instance >= (int)c->inst.size()) return TEUK_EINVAL;
    if (step) *step = c->inst[instance].step;
    if (dt) *dt = c->inst[instance].dt;
    return TEUK_OK;
}

extern "C" teuk_status teuk_get_geometry(const teuk_ctx* c, int instance, double* out);

extern "C" teuk_status teuk_set_tiling(teuk_ctx* c, int strip, int steps_per_launch) {
    if (!c) return TEUK_EINVAL;
    if (strip < 0 || steps_per_launch < 0)
        TK_FAIL(c, TEUK_EINVAL, "tiling parameters must be >= 0");
    c->strip = strip;
    c->steps_per_launch = steps_per_launch;
    invalidate_graph(c);
    return refresh_partitions(c);
}

extern "C" teuk_status teuk_set_fault_injection(teuk_ctx* c, int64_t skip_release_item,
                                                long long spin_limit) {
    if (!c) return TEUK_EINVAL;
    if (spin_limit < 0) TK_FAIL(c, TEUK_EINVAL, "spin_limit must be >= 0");
    c->inject_skip_item = skip_release_item;
    c->spin_limit = spin_limit > 0 ? spin_limit : 20000000LL;
    invalidate_graph(c);
    return TEUK_OK;
}

extern "C" teuk_status teuk_set_fill_fault(teuk_ctx* c, int instance, int column) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    c->inst[instance].fault_col = column < 0 ? -1 : column;
    invalidate_graph(c);
    return TEUK_OK;
}

extern "C" teuk_status teuk_set_instance_tiling(teuk_ctx* c, int instance, int strip) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    if (strip < 0) TK_FAIL(c, TEUK_EINVAL, "strip must be >= 0");
    c->inst[instance].strip = strip;
    invalidate_graph(c);
    return refresh_partition(c, c->inst[instance]);
}

// Contexts that step through the persistent kernels (several instances, or one in
// persistent mode) run one launch per block-size class over all its instances, so a
// strip length is evaluated in that setting: trial_steps steps of the whole context are
// timed for each candidate, first with one length for every instance, then class by
// class with the others held at their best, on the live state; afterwards every
// instance's state, time level and waveform records are restored from a snapshot.
// (Timing one instance alone favours short strips, which fill the GPU with one
// instance but, in the batch, pay the ring's start-up every few columns.)
static teuk_status autotune_batched(teuk_ctx* c, int trial_steps, int* chosen) {
    const int ni = (int)c->inst.size();
    struct Snap {
        void* st[2] = {nullptr, nullptr};
        double2* wave = nullptr;
        int64_t step = 0, lo = 0, hi = 0;
        int cur = 0;
    };
    std::vector<Snap> snap(ni);
    auto release = [&]() {
        for (Snap& q : snap) {
            for (void* p : q.st)
                if (p) dfree(c, p, c->stream);
            if (q.wave) dfree(c, q.wave, c->stream);
        }
    };
    teuk_status err = TEUK_OK;
    for (int k = 0; k < ni && !err; ++k) {
        Instance& I = c->inst[k];
        const int nplanes = I.p.prec == TEUK_FP32 ? 1 : 2;
        Snap& q = snap[k];
        q.step = I.step;
        q.cur = I.cur;
        q.lo = I.wave_lo;
        q.hi = I.wave_hi;
        for (int pl = 0; pl < nplanes && !err; ++pl) {
            if (dmalloc(c, &q.st[pl], I.plane_bytes, c->stream) != cudaSuccess) err = TEUK_ENOMEM;
            else cudaMemcpyAsync(q.st[pl], I.state[I.cur][pl], I.plane_bytes, cudaMemcpyDeviceToDevice, c->stream);
        }
        const size_t wb = sizeof(double2) * (size_t)I.wave_cap * (size_t)I.p.n_theta;
        if (!err) {
            if (dmalloc(c, (void**)&q.wave, wb, c->stream) != cudaSuccess) err = TEUK_ENOMEM;
            else cudaMemcpyAsync(q.wave, I.wave, wb, cudaMemcpyDeviceToDevice, c->stream);
        }
    }
    if (err) {
        release();
        cudaGetLastError();
        TK_FAIL(c, err, "autotune: snapshot allocation failed");
    }
    cudaEvent_t e0, e1;
    TK_CUDA(c, cudaEventCreate(&e0));
    TK_CUDA(c, cudaEventCreate(&e1));
    auto trial = [&](float& ms) -> teuk_status {
        teuk_status st = batched_step(c, trial_steps);   // warm-up (and graph capture)
        if (st) return st;
        cudaEventRecord(e0, c->stream);
        st = batched_step(c, trial_steps);
        if (st) return st;
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return TEUK_ECUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        return TEUK_OK;
    };
    auto set_strip = [&](const std::vector<int>& members, int L) {
        for (int k : members) c->inst[k].strip = std::max(1, std::min(L, c->inst[k].p.n_rstar - 2));
    };
    // block-size classes, as batched_step forms them (instances with the same pitch)
    std::vector<std::vector<int>> cls;
    std::vector<int> cls_pitch, all(ni);
    for (int k = 0; k < ni; ++k) {
        all[k] = k;
        int q = 0;
        while (q < (int)cls.size() && cls_pitch[q] != c->inst[k].pitch) ++q;
        if (q == (int)cls.size()) {
            cls.emplace_back();
            cls_pitch.push_back(c->inst[k].pitch);
        }
        cls[q].push_back(k);
    }
    // strips of 16 to 512 columns; shorter ones as well when 16-column strips would leave
    // fewer than four work items per step for each SM (a grid too small to fill the GPU,
    // where one-column strips are fastest)
    std::vector<int> cand = {16, 32, 64, 128, 256, 512};
    {
        int64_t items16 = 0;
        for (int k = 0; k < ni; ++k) items16 += (c->inst[k].p.n_rstar - 2 + 15) / 16;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (items16 < 4 * (int64_t)(sms > 0 ? sms : 1)) cand.insert(cand.begin(), {1, 2, 4, 8});
    }
    float best_ms = 1e30f;
    int best_all = 128;
    teuk_status st = TEUK_OK;
    for (int L : cand) {
        set_strip(all, L);
        float ms = 0.f;
        if ((st = trial(ms))) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_all = L;
        }
    }
    set_strip(all, best_all);
    if (!st && cls.size() > 1) {
        for (const std::vector<int>& members : cls) {
            int best_c = best_all;
            for (int L : cand) {
                if (L == best_all) continue;
                set_strip(members, L);
                float ms = 0.f;
                if ((st = trial(ms))) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_c = L;
                }
            }
            set_strip(members, best_c);
            if (st) break;
        }
    }
    // restore the state, time level and waveform records of every instance
    for (int k = 0; k < ni; ++k) {
        Instance& I = c->inst[k];
        const Snap& q = snap[k];
        const int nplanes = I.p.prec == TEUK_FP32 ? 1 : 2;
        for (int pl = 0; pl < nplanes; ++pl)
            cudaMemcpyAsync(I.state[q.cur][pl], q.st[pl], I.plane_bytes, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(I.wave, q.wave, sizeof(double2) * (size_t)I.wave_cap * (size_t)I.p.n_theta,
                        cudaMemcpyDeviceToDevice, c->stream);
        I.step = q.step;
        I.cur = q.cur;
        I.wave_lo = q.lo;
        I.wave_hi = q.hi;
        if (chosen) chosen[k] = I.strip;
    }
    release();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    invalidate_graph(c);
    if (st) return st;
    TK_CUDA(c, cudaStreamSynchronize(c->stream));
    return refresh_partitions(c);
}

// Single instance stepped one launch per step: time each candidate strip length on a
// scratch copy of the instance and keep the fastest.  Otherwise see autotune_batched.
extern "C" teuk_status teuk_autotune(teuk_ctx* c, int trial_steps, int* chosen) {
    if (!c) return TEUK_EINVAL;
    if (trial_steps < 1) TK_FAIL(c, TEUK_EINVAL, "trial_steps must be >= 1");
    if (c->inst.size() > 1 || c->steps_per_launch == 0) return autotune_batched(c, trial_steps, chosen);
    const int ni = (int)c->inst.size();
    std::vector<int> best(ni, 0), best_res(ni, 0);
    cudaEvent_t e0, e1;
    TK_CUDA(c, cudaEventCreate(&e0));
    TK_CUDA(c, cudaEventCreate(&e1));
    for (int k = 0; k < ni; ++k) {
        if (best[k]) continue;
        Instance& I = c->inst[k];
        auto bucket = [](int nr) { int b = 0; while ((1 << b) < nr) ++b; return b; };
        const int nplanes = I.p.prec == TEUK_FP32 ? 1 : 2;
        void* scr[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
        double2* scr_wave = nullptr;
        teuk_status err = TEUK_OK;
        for (int b = 0; b < 2 && !err; ++b)
            for (int q = 0; q < nplanes && !err; ++q)
                if (dmalloc(c, &scr[b][q], I.plane_bytes, c->stream) != cudaSuccess) err = TEUK_ENOMEM;
        if (!err && dmalloc(c, (void**)&scr_wave, sizeof(double2) * I.p.n_theta * (trial_steps + 2),
                                    c->stream) != cudaSuccess)
            err = TEUK_ENOMEM;
        float best_ms = 1e30f;
        int best_strip = auto_strip(I);
        if (!err) {
            InstDev d = dev_of(c, I);
            d.wave = scr_wave;           // trial records must not touch the live ring
            d.wave_cap = trial_steps + 2;
            for (int q = 0; q < nplanes; ++q) {
                cudaMemcpyAsync(scr[0][q], I.state[I.cur][q], I.plane_bytes, cudaMemcpyDeviceToDevice,
                                c->stream);
                d.buf[0][q] = scr[0][q];
                d.buf[1][q] = scr[1][q];
            }
            const int cand[] = {1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};
            for (int ch : cand) {
                if (ch > I.p.n_rstar - 2) break;
                for (int w = 0; w < 2; ++w) launch_step(c->stream, d, I.step + w, w & 1, ch);
                cudaEventRecord(e0, c->stream);
                for (int t = 0; t < trial_steps; ++t) launch_step(c->stream, d, I.step + t, t & 1, ch);
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                c->launches += trial_steps + 2;
                if (ms < best_ms) { best_ms = ms; best_strip = ch; }
            }
            // resident launches, halo 1 .. 4 (circular orbits; a moving particle is stepped
            // one launch per step)
            // (halo 1 .. 4, aiming at 1 .. 3 blocks per SM; a plan equal to one already
            // timed is skipped; best_res holds halo + 16 (blocks per SM - 1))
            for (int code = 1; code <= 4 + 16 * 2 && !(I.src_on && I.sd.moving); ++code) {
                const int hh = code % 16, bps = code / 16 + 1;
                if (hh < 1 || hh > 4) continue;
                ResidentPlan plan;
                if (!resident_plan(I.p.prec, I.p.n_rstar, I.pitch, hh, bps, &plan)) continue;
                if (bps > 1) {
                    ResidentPlan fewer;
                    if (resident_plan(I.p.prec, I.p.n_rstar, I.pitch, hh, bps - 1, &fewer) && fewer.nb == plan.nb)
                        continue;
                }
                unsigned char* xg = nullptr;
                int* fl = nullptr;
                const size_t xg_bytes = (size_t)nplanes * 2 * plan.nb * 2 * hh * I.pitch * 16;
                if (dmalloc(c, (void**)&xg, xg_bytes, c->stream) == cudaSuccess &&
                    dmalloc(c, (void**)&fl, sizeof(int) * kResFlagStride * (plan.nb + 1), c->stream) == cudaSuccess) {
                    ResidentArgs a{};
                    a.d = d;
                    a.step0 = I.step;
                    a.bin = 0;
                    a.h = hh;
                    a.nb = plan.nb;
                    a.xg = xg;
                    a.flags = fl;
                    a.abort = fl + (size_t)kResFlagStride * plan.nb;
                    a.skip_publish = -1;
                    float ms = 1e30f;
                    bool ok = true;
                    for (int w = 0; w < 2 && ok; ++w) {   // warm-up (2 steps), then the timed run
                        a.n = w == 0 ? 2 : trial_steps;
                        a.obin = (int)(a.n & 1);
                        cudaMemsetAsync(fl, 0, sizeof(int) * kResFlagStride * (plan.nb + 1), c->stream);
                        if (w == 1) cudaEventRecord(e0, c->stream);
                        ok = launch_resident(c->stream, a, plan) == cudaSuccess;
                        if (w == 1) cudaEventRecord(e1, c->stream);
                    }
                    if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                    c->launches += 2;
                    if (ok && ms < best_ms) {
                        best_ms = ms;
                        best_res[k] = code;
                    }
                }
                cudaGetLastError();
                if (xg) dfree(c, xg, c->stream);
                if (fl) dfree(c, fl, c->stream);
            }
        }
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 2; ++q)
                if (scr[b][q]) dfree(c, scr[b][q], c->stream);
        if (scr_wave) dfree(c, scr_wave, c->stream);
        if (err) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            TK_FAIL(c, err, "autotune: scratch allocation failed");
        }
        for (int k2 = k; k2 < ni; ++k2) {
            Instance& J = c->inst[k2];
            if (J.p.n_theta == I.p.n_theta && J.p.prec == I.p.prec &&
                bucket(J.p.n_rstar) == bucket(I.p.n_rstar) && !best[k2])
                best[k2] = best_strip;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int k = 0; k < ni; ++k) {
        c->inst[k].strip = best[k];
        teuk_status st = set_resident(c, c->inst[k], best_res[k] % 16, best_res[k] / 16 + 1);
        if (st) return st;
        if (chosen) chosen[k] = best_res[k] > 0 ? -best_res[k] : best[k];
    }
    invalidate_graph(c);
    TK_CUDA(c, cudaGetLastError());
    return refresh_partitions(c);
}

extern "C" int64_t teuk_kernel_launches(const teuk_ctx* c) { return c ? c->launches : 0; }

extern "C" void teuk_destroy(teuk_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);   // no replay of the context's graphs is in flight
    {
        if (c->sum_buf) dfree(c, c->sum_buf, c->stream);
        Batch& B = c->batch;
        if (B.exec) cudaGraphExecDestroy(B.exec);
        if (B.graph) cudaGraphDestroy(B.graph);
        void* ptrs[] = {B.d_blob, B.d_abort};
        for (void* q : ptrs)
            if (q) dfree(c, q, c->stream);
        for (BatchClass& K : B.cls) {
            if (K.d_counter) dfree(c, K.d_counter, c->stream);
            if (K.d_flags) dfree(c, K.d_flags, c->stream);
        }
    }
    for (Instance& I : c->inst) free_instance(c, I);
    if (c->status) dfree(c, c->status, c->stream);
    cudaStreamSynchronize(c->stream);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

extern "C" const char* teuk_last_error(const teuk_ctx* c) {
    return c ? c->err.c_str() : g_create_err.c_str();
}

// ------------------------------------------------------------------ adjoint

namespace {

// r(r*) on the host (the extraction radius of the built-in loss): safeguarded Newton
// in y = ln(r - r_+), the same inversion of Eq. (2) the setup kernel performs.
double r_of_rstar_host(double M, double a, double target) {
    double d = std::sqrt(M * M - a * a), rp = M + d, rm = M - d;
    double k = 2.0 * M / (rp - rm);
    auto rs = [&](double x) {
        double r = rp + x;
        return r + k * rp * std::log(x / (2.0 * M)) - k * rm * std::log((r - rm) / (2.0 * M));
    };
    double lo = -700.0, hi = 30.0;
    double y = target > rp + 4.0 ? std::log(target) : (target - rp) / (k * rp);
    y = std::fmin(std::fmax(y, lo + 1.0), hi - 1.0);
    for (int it = 0; it < 200; ++it) {
        double x = std::exp(y), f = rs(x) - target;
        if (f > 0.0) hi = y; else lo = y;
        double r = rp + x;
        double yn = y - f / ((r * r + a * a) / (x + rp - rm));
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
        if (std::fabs(yn - y) <= 1e-15 * std::fmax(1.0, std::fabs(y))) { y = yn; break; }
        y = yn;
    }
    return rp + std::exp(y);
}

// Device buffers of one adjoint call, released in reverse order of allocation.
struct AdjBuffers {
    const teuk_ctx* c;
    cudaStream_t st;
    std::vector<void*> ptrs;
    AdjBuffers(const teuk_ctx* cc, cudaStream_t s) : c(cc), st(s) {}
    cudaError_t get(void** p, size_t bytes) {
        cudaError_t e = dmalloc(c, p, bytes, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~AdjBuffers() {
        for (void* q : ptrs) dfree(c, q, st);
    }
};

}  // namespace

extern "C" teuk_status teuk_get_geometry(const teuk_ctx* c, int instance, double* out) {
    if (!c || !out || instance < 0 || instance >= (int)c->inst.size()) return TEUK_EINVAL;
    const Instance& I = c->inst[instance];
    out[0] = I.drs; out[1] = I.dth; out[2] = I.dt; out[3] = I.rp; out[4] = I.rm;
    out[5] = r_of_rstar_host(I.p.M, I.p.a, I.p.rstar_ext);
    out[6] = (double)I.i_e; out[7] = I.f_e;
    return TEUK_OK;
}

extern "C" teuk_status teuk_slab_halo_bytes(const teuk_ctx* c, int instance, int64_t* bytes) {
    if (!c || !bytes || instance < 0 || instance >= (int)c->inst.size()) return TEUK_EINVAL;
    const Instance& I = c->inst[instance];
    const int planes = I.p.prec == TEUK_FP32 ? 1 : 2;
    *bytes = (int64_t)planes * I.pitch * 16;
    return TEUK_OK;
}

namespace {
// Device copy of local column col of the current level to / from dev (planes one after
// the other, pitch 16-byte nodes each), on the context's stream.
teuk_status column_copy(teuk_ctx* c, Instance& I, int col, void* dev, bool out) {
    const int planes = I.p.prec == TEUK_FP32 ? 1 : 2;
    const size_t cb = (size_t)I.pitch * 16;
    for (int k = 0; k < planes; ++k) {
        char* st = (char*)I.state[I.cur][k] + (size_t)col * cb;
        char* ex = (char*)dev + k * cb;
        TK_CUDA(c, cudaMemcpyAsync(out ? ex : st, out ? st : ex, cb, cudaMemcpyDeviceToDevice, c->stream));
    }
    return TEUK_OK;
}
}  // namespace

extern "C" teuk_status teuk_slab_export(teuk_ctx* c, int instance, int side, void* dev_buf) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    Instance& I = c->inst[instance];
    if (!I.slab || (side != 0 && side != 1) || !dev_buf)
        TK_FAIL(c, TEUK_EINVAL, "need a slab instance, side 0 or 1 and a device buffer");
    return column_copy(c, I, side == 0 ? 1 : I.p.n_rstar - 2, dev_buf, true);
}

extern "C" teuk_status teuk_slab_import(teuk_ctx* c, int instance, int side, const void* dev_buf) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    Instance& I = c->inst[instance];
    if (!I.slab || (side != 0 && side != 1) || !dev_buf)
        TK_FAIL(c, TEUK_EINVAL, "need a slab instance, side 0 or 1 and a device buffer");
    st = column_copy(c, I, side == 0 ? 0 : I.p.n_rstar - 1, (void*)dev_buf, false);
    if (st) return st;
    // the record of the current level, if it reads the column just replaced
    const int col = side == 0 ? 0 : I.p.n_rstar - 1;
    if (I.ext_here && (I.i_e == col || I.i_e + 1 == col) && I.wave_hi > I.wave_lo) {
        launch_extract(c->stream, dev_of(c, I), I.step, I.cur);
        c->launches++;
        TK_CUDA(c, cudaGetLastError());
    }
    return TEUK_OK;
}

extern "C" teuk_status teuk_adjoint_n(teuk_ctx* c, int instance, int64_t step0, int64_t n,
                                      int64_t ckpt_every, const double* grad_wave,
                                      double* grad_amps, double* grad_r0, double* loss) {
    teuk_status st = check_instance(c, instance);
    if (st) return st;
    Instance& I = c->inst[instance];
    if (n < 1 || step0 < 0) TK_FAIL(c, TEUK_EINVAL, "need n >= 1 and step0 >= 0");
    if (I.sd.moving)
        TK_FAIL(c, TEUK_EINVAL, "source gradients are defined for the circular-orbit source only");
    if (I.slab) TK_FAIL(c, TEUK_EINVAL, "the adjoint is not available for slab instances");
    const bool builtin = grad_wave == nullptr;
    if (builtin && I.step != step0)
        TK_FAIL(c, TEUK_ESTATE, "built-in loss: the state is at step %lld, not step0 = %lld",
                (long long)I.step, (long long)step0);
    cudaStream_t s = c->stream;
    const int nth = I.p.n_theta;
    if (I.p.prec == TEUK_FP64 || I.p.prec == TEUK_FP64_DF) {   // (FP32 instances form theirs)
        st = coef_tables(c, I);
        if (st) return st;
    }
    // co-state planes ([nr][pitch] complex): FP64 for FP64 instances, else FP32 with
    // compensation planes for lam
    const bool co32 = I.p.prec == TEUK_FP32 || I.p.prec == TEUK_FP32_KAHAN;
    const size_t plane = (size_t)I.p.n_rstar * I.pitch * (co32 ? sizeof(float2) : sizeof(double2));
    AdjBuffers B(c, s);
    CoLevel lam[2] = {};
    for (int b = 0; b < 2; ++b) {
        TK_CUDA(c, B.get(&lam[b].F, plane));
        TK_CUDA(c, B.get(&lam[b].P, plane));
        if (co32) {
            TK_CUDA(c, B.get(&lam[b].Fc, plane));
            TK_CUDA(c, B.get(&lam[b].Pc, plane));
        }
    }
    // the fused reverse step's strip; with a source, a ring of window co-states that
    // adj_src_grad_kernel turns into gradients every `slots` steps (32 MB at most)
    int adj_strip = 0;
    adj_step_plan(dev_of(c, I), &adj_strip);
    const bool src_on = I.src_on;
    const size_t wbytes = src_on ? adj_window_bytes(dev_of(c, I)) : 0;
    const int64_t slots = src_on ? std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(n, 256),
                                                                          (int64_t)((32u << 20) / wbytes)))
                                 : 0;
    char* wring = nullptr;
    if (src_on) TK_CUDA(c, B.get((void**)&wring, wbytes * (size_t)slots));
    const size_t wh_bytes = (size_t)I.sd.nh * I.sd.nj * (co32 ? sizeof(float2) : sizeof(double2));
    double *gA = nullptr, *gR = nullptr, *lossrec = nullptr, *scal = nullptr;
    double2* gbar = nullptr;
    TK_CUDA(c, B.get((void**)&gA, sizeof(double) * n));
    TK_CUDA(c, B.get((void**)&gR, sizeof(double) * n));
    TK_CUDA(c, B.get((void**)&scal, sizeof(double) * 3));
    // record cotangents: all n, or (checkpointed built-in loss) a ring of one segment's
    const int64_t Kc = (builtin && ckpt_every > 0) ? std::min<int64_t>(ckpt_every, n) : n;
    const int64_t gcap = (builtin && ckpt_every > 0) ? Kc + 1 : n;
    TK_CUDA(c, B.get((void**)&gbar, sizeof(double2) * nth * (size_t)gcap));
    auto gslot = [&](int64_t idx) { return gbar + (size_t)(idx % gcap) * nth; };
    TK_CUDA(c, cudaMemsetAsync(gA, 0, sizeof(double) * n, s));
    TK_CUDA(c, cudaMemsetAsync(gR, 0, sizeof(double) * n, s));
    TK_CUDA(c, cudaMemsetAsync(scal, 0, sizeof(double) * 3, s));
    InstDev d = dev_of(c, I);
    double r6 = 0.0;
    // forward-sweep helpers ------------------------------------------------
    // run `count` steps on the buffers of dv (which start in buffer cur), recording
    // levels into the ring of dv; returns the buffer holding the result.
    auto forward = [&](InstDev dv, int cur, int64_t level, int64_t count, int strip) {
        cur = run_steps(c, I, dv, s, cur, level, count, strip);
        launch_extract(s, dv, level + count, cur);
        c->launches++;
        return cur;
    };
    const int strip = eff_strip(c, I);
    // the segment plan: segments [a_k, a_k + len_k) of the steps step0 .. step0+n-1
    const int64_t K = Kc;
    int64_t nseg = (n + K - 1) / K;
    void* ckpt = nullptr;
    void* scratch_state[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    double2* segrec = nullptr;
    const int nplanes = I.p.prec == TEUK_FP32 ? 1 : 2;
    if (builtin) {
        r6 = std::pow(r_of_rstar_host(I.p.M, I.p.a, I.p.rstar_ext), 6);
        TK_CUDA(c, B.get((void**)&lossrec, sizeof(double) * n));
        TK_CUDA(c, B.get((void**)&segrec, sizeof(double2) * nth * (size_t)(K + 1)));
        if (ckpt_every > 0) {
            TK_CUDA(c, B.get(&ckpt, I.plane_bytes * nplanes * (size_t)nseg));
            for (int b = 0; b < 2; ++b)
                for (int k = 0; k < nplanes; ++k)
                    TK_CUDA(c, B.get(&scratch_state[b][k], I.plane_bytes));
        }
        // forward sweep on the context's own state, checkpointing each segment start
        InstDev fw = d;
        fw.wave = segrec;
        fw.wave_cap = K + 1;
        for (int64_t sg = 0; sg < nseg; ++sg) {
            int64_t a = step0 + sg * K, len = std::min(K, n - sg * K);
            if (ckpt)
                for (int k = 0; k < nplanes; ++k)
                    TK_CUDA(c, cudaMemcpyAsync((char*)ckpt + ((size_t)sg * nplanes + k) * I.plane_bytes,
                                               I.state[I.cur][k], I.plane_bytes,
                                               cudaMemcpyDeviceToDevice, s));
            fw = dev_of(c, I);
            fw.wave = segrec;
            fw.wave_cap = K + 1;
            I.cur = forward(fw, I.cur, a, len, strip);
            I.step = a + len;
            if (!ckpt) {  // one segment holds everything: take the loss now
                launch_loss_records(s, segrec, K + 1, nth, a + 1, len, r6, lossrec + (a - step0),
                                    gbar, gcap, a - step0);
                c->launches++;
            }
        }
        I.wave_lo = I.wave_hi = I.step;  // the forward records went to the adjoint's own buffer
    } else {
        TK_CUDA(c, cudaMemcpyAsync(gbar, grad_wave, sizeof(double2) * nth * (size_t)n,
                                   cudaMemcpyHostToDevice, s));
    }
    // reverse sweep ----------------------------------------------------------
    int cur = 0;
    bool started = false;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        int64_t a = step0 + sg * K, len = std::min(K, n - sg * K);
        if (builtin && ckpt) {
            // recompute this segment's waveform from its checkpoint
            InstDev rv = d;
            for (int k = 0; k < nplanes; ++k) {
                rv.buf[0][k] = scratch_state[0][k];
                rv.buf[1][k] = scratch_state[1][k];
                TK_CUDA(c, cudaMemcpyAsync(scratch_state[0][k],
                                           (char*)ckpt + ((size_t)sg * nplanes + k) * I.plane_bytes,
                                           I.plane_bytes, cudaMemcpyDeviceToDevice, s));
            }
            rv.wave = segrec;
            rv.wave_cap = K + 1;
            forward(rv, 0, a, len, strip);
            // records a+1 .. a+len, and also record a (the last record of the previous
            // segment), which this segment's first reverse step needs before the
            // previous segment is recomputed; writing it twice stores the same value
            int64_t lo = a > step0 ? a : a + 1;
            launch_loss_records(s, segrec, K + 1, nth, lo, a + len - lo + 1, r6,
                                lossrec + (lo - step0 - 1), gbar, gcap, lo - step0 - 1);
            c->launches++;
        }
        for (int64_t m = a + len - 1; m >= a; --m) {
            const int64_t k = m - step0;  // step index within the call
            if (!started) {
                launch_adj_init(s, d, gslot(n - 1), lam[cur]);
                c->launches++;
                started = true;
            }
            const double2* gb = k >= 1 ? gslot(k - 1) : nullptr;
            char* slot = src_on ? wring + (size_t)(k % slots) * wbytes : nullptr;
            launch_adj_step(s, d, lam[cur], gb, lam[1 - cur], adj_strip, slot, slot ? slot + wh_bytes : nullptr);
            if (src_on && k % slots == 0) {   // the steps k .. k + slots - 1 are all stored
                launch_adj_src_grad(s, d, step0, k, std::min<int64_t>(n - 1, k + slots - 1) - k + 1,
                                    (int)slots, wring, gA, gR);
                c->launches++;
            }
            c->launches++;
            cur = 1 - cur;
        }
    }
    launch_ordered_sum(s, gR, n, scal + 0);
    c->launches++;
    if (builtin) {
        launch_ordered_sum(s, lossrec, n, scal + 1);
        c->launches++;
    }
    TK_CUDA(c, cudaGetLastError());
    double h[3] = {0, 0, 0};
    TK_CUDA(c, cudaMemcpyAsync(h, scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    if (grad_amps)
        TK_CUDA(c, cudaMemcpyAsync(grad_amps, gA, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    TK_CUDA(c, cudaStreamSynchronize(s));
    if (grad_r0) *grad_r0 = h[0];
    if (loss && builtin) *loss = h[1];
    return TEUK_OK;
}
