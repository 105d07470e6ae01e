// teuk_internal.cuh -- device-side data structures shared by the library's kernels.
//
// HBM layout of one instance (theta is the fastest index; each r* column of n_theta
// nodes is padded to a pitch that is a multiple of 32 elements, so a column starts on
// a 512-byte boundary and one thread block reads it in one coalesced sweep):
//   state   two ping-pong buffers, each made of "planes" [n_rstar][pitch]:
//             FP64        plane 0 = Phi (double2), plane 1 = Pi (double2)
//             FP32        plane 0 = {Phi_R, Phi_I, Pi_R, Pi_I} (float4)
//             FP32_KAHAN  plane 0 = hi {Phi, Pi} (float4), plane 1 = c {Phi, Pi} (float4),
//                         the represented value being hi - c
//             FP64_DF     plane 0 = hi {Phi, Pi} (float4), plane 1 = lo {Phi, Pi} (float4),
//                         the value being hi + lo (double-float)
//   coef_h  [9][n_rstar][pitch] FP64 (double) and FP64_DF ((hi, lo) float pairs) paths:
//           predictor coefficients at half nodes (i+1/2, j)
//   coef_i  [9][n_rstar][pitch] the same at integer nodes (i, j)
//   source  FP64 complex profile on a window of nodes around the particle
//   wave    FP64 ring of waveform records [capacity][n_theta] (double2)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace teuk {

constexpr int kNCoef = 9;        // coefficients per node and sub-step
constexpr int kPitchAlign = 32;  // elements

// Coefficient planes (same order at half and integer nodes; "s" is 1/2 for the
// predictor and 1 for the corrector, i.e. the fraction of dt of the sub-step):
//   0: g    = s dt b / dr*                       (D term of Eqs. 13-14)
//   1,2: E1 = -s dt c_t                          (Pi coefficient of S_Pi)
//   3,4: E2 = s dt P* / dr*,  P* = c_t b + p* - b b_{,r*}
//   5:   ep = s dt w (1/dth^2 + cot/(2 dth))     (forward theta difference)
//   6:   em = s dt w (1/dth^2 - cot/(2 dth))     (backward theta difference)
//   7,8: E3 = s dt (q - w V)                     (zero-order term)
enum CoefIdx { C_G = 0, C_E1R, C_E1I, C_E2R, C_E2I, C_EP, C_EM, C_E3R, C_E3I };

struct SourceDev {
    int on;
    // integer nodes i in [i_lo, i_lo + ni), half nodes i+1/2 in [h_lo, h_lo + nh),
    // rows j in [j_lo, j_lo + nj)
    int i_lo, ni, h_lo, nh, j_lo, nj;
    const double2* P_int;    // [nj][ni]   profile P (no phase)
    const double2* P_half;   // [nj][nh]
    const double2* dP_int;   // [nj][ni]   dP/dr0
    const double2* dP_half;  // [nj][nh]
    // P again for the step kernels: column-major ([ni][q_stride], [nh][q_stride]) so that
    // the rows of one column are contiguous, in the state's arithmetic type (double2 on
    // the FP64 path, float2 on the FP32 paths); q_stride >= nj makes every column a
    // 16-byte aligned multiple of 16 bytes (the step kernel prefetches columns into L2)
    const void* Q_int;
    const void* Q_half;
    int q_stride;
    double omega, phase0;    // tau = A_n exp(-i (omega t + phase0)) P
    double domega, dphase0;  // d omega/d r0, d phase0/d r0
    const double* amps;      // A_n for n < n_amps, else 1
    int64_t n_amps;
    // Moving particle (a sampled path, teuk_set_trajectory): the window bounds the whole
    // path, Q holds the static prefactor pref / (2 pi sig_r sig_th) and the source of
    // step n at node (i, j) is  fac g_r[n](i) g_th[n](j) Q(i, j),  fac = dt_sub A e^{-i m phi_p}
    // of sample 2n (predictor, half nodes) or 2n + 1 (corrector, integer nodes).
    int moving;
    int64_t n_traj;          // steps with tables; later steps have no source
    const double2* amp;      // [n_traj][2] A e^{-i m phi_p} of samples 2n, 2n + 1 (0: no sample)
    const void* gr;          // [n_traj][nh + ni] radial factors, half nodes then integer
                             // nodes, in the arithmetic type (double, float or DF)
    const void* gt;          // [n_traj][2][nj] angular factors of samples 2n, 2n + 1
};

// FP32 paths form their coefficients in registers from 1D tables (rounded from FP64 at
// setup), instead of reading 2D tables every step.  The entry of radial column i holds
// the values of the half node i+1/2 in .x (sub-step fraction s = 1/2) and of the node i
// in .y (s = 1), so that both coefficient sets of a column are formed together in
// paired FP32 instructions.  With sdt = s dt:
//   Sigma^2 = R2 + naD sin^2 (naD = -a^2 Delta),  iS = 1/Sigma^2,  rs = Sigma^{-1}
//   g  = Rd * rs                                      (Rd = sdt R / dr*)
//   c_t = (ctr iS, (cti + ctc cos) iS),  E1 = nsdt c_t   (nsdt = -sdt)
//   E2 = c_t g + ((pr + nbb sin^2 iS) iS, pi iS)       (pr, pi, nbb = -bb scaled by sdt/dr*)
//   A, B = Ds iS / dth^2, Ds iS cot / (2 dth)         (Ds = sdt Delta; the split angular
//                                                       form, ep = A + B, em = A - B)
//   E3 = ((qr + nDs V) iS, qi iS)                      (qr, qi scaled by sdt; nDs = -Ds)
struct RTab2 { float2 R2, naD, Rd, ctr, cti, ctc, pr, pi, nbb, Ds, nDs, qr, qi, nsdt, pad0, pad1; };
// Per theta row: sin^2, cos, V = (m + s cos)^2/sin^2 - s, i2 = 1/dth^2, i1 = cot/(2 dth)
struct ThTab { float sin2, cs, V, i2, i1, pad0, pad1, pad2; };

struct InstDev {
    int nr, nth, pitch, prec;
    double drs, dth, dt;
    float ghost_f;            // +1 even |m + s|, -1 odd |m + s|
    double ghost;
    void* buf[2][2];          // [ping-pong buffer][plane]
    const void* coef_h;       // [9][nr][pitch] (double or float)
    const void* coef_i;
    const RTab2* rtab;        // [nr] FP32 paths: radial tables (half node, node) per column
    const ThTab* thtab;       // [nth]
    SourceDev src;
    int i_e;                  // extraction between i_e and i_e + 1
    double f_e;
    double2* wave;            // [wave_cap][nth]
    int64_t wave_cap;
    unsigned int* status;     // device status word (bit flags)
    int fault_col;            // testing aid: this input column is never filled into the
                              // step kernels' ring (-1: none)
    const int64_t* step_base; // per-step kernels replayed from a graph: their step argument
                              // is an offset from *step_base (null: the argument is the step)
};

enum StatusBits : unsigned int { ST_NONFINITE = 1u, ST_TIMEOUT = 2u, ST_BOUNDS = 4u };

// Checked builds (-DTEUK_CHECK, libteuk_check.so): TK_IN(status, i, n) tests an index
// against the extent of the buffer it is about to address; a failure sets ST_BOUNDS in
// the status word and the caller skips the access (a load gives zero), so nothing traps
// and teuk_sync reports TEUK_EBOUNDS.  Release builds compile every check to `true`.
#ifdef TEUK_CHECK
__device__ __forceinline__ bool check_index(unsigned int* status, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(status, (unsigned)ST_BOUNDS);
    return false;
}
#define TK_IN(status, i, n) ::teuk::check_index((status), (long long)(i), (long long)(n))
#else
#define TK_IN(status, i, n) true
#endif

// Batched persistent launch over many instances of one block-size class (teuk_step.cu).
// Work items are (relative step s, instance k, r* strip) in that order of priority;
// items of one step are numbered instance by instance from item_base[k].
struct BatchDev {
    const InstDev* inst;        // [n_inst] descriptors of this call
    const int64_t* item_base;   // [n_inst + 1] first item of each instance within a step
    const int* strip;           // [n_inst] r* columns per item
    const int* nstrip;          // [n_inst] items per instance and step
    const int64_t* base_step;   // [n_inst] time level at the start of the call
    const int* base_bin;        // [n_inst] buffer holding that level
    const int64_t* n_steps;     // steps of this call (device scalar)
    int n_inst;
    int64_t items_per_step;
    unsigned long long* counter;  // next work item
    int* flags;                 // [items_per_step] relative steps completed by each item
    int* abort;                 // set when a wait gives up: everyone stops
    unsigned int* status;
    long long spin_limit;       // polls before a wait gives up
    int64_t skip_release_item;  // testing aid (-1: none): this item of relative step 0 never
                                // releases its flag, so its neighbours' waits run out
};

// One cooperative launch of the resident kernel (teuk_resident.cu): n steps of one
// instance held in shared memory, exchanging h boundary columns with the neighbouring
// blocks every h steps.
struct ResidentArgs {
    InstDev d;
    int64_t step0;        // time level at the start
    int bin, obin;        // buffer holding it, buffer receiving the final level
    int64_t n;            // steps
    int h;                // halo width = steps between exchanges
    int nb;               // blocks
    unsigned char* xg;    // exchange slots [planes][2][nb][2][h][pitch] 16-byte nodes
    int* flags;           // [nb][kResFlagStride] 1 + exchanges published, one 128-byte line
                          // a block (zeroed before each launch)
    int* abort;           // set when a wait gives up
    int skip_publish;     // testing aid (-1: none): this block never publishes its exchanges,
                          // so its neighbours' waits run out
    int no_wait;          // blocked launches (n <= h, obin != bin): no exchange and no wait
                          // before the final level is written (no block reads buffer obin)
};
constexpr int kResFlagStride = 32;   // ints between two blocks' flags (a 128-byte line each)
// Launch shape of the resident kernel for one instance.
struct ResidentPlan { int nb = 0, threads = 0, h = 0, bps = 1; size_t smem = 0; };

__host__ __device__ inline size_t plane_elems(const InstDev& d) {
    return (size_t)d.nr * (size_t)d.pitch;
}

// Offset of node (i, j) = (r*_i, theta_j) in a plane.
__host__ __device__ inline size_t node_index(const InstDev& d, int i, int j) {
    return (size_t)i * (size_t)d.pitch + (size_t)j;
}

// ---- host launchers (each defined next to its kernels) ----
// teuk_setup.cu
// (off: node k of the instance is node k + off of its grid, > 0 for a slab)
void launch_invert_tortoise(cudaStream_t st, double M, double a, double rstar_min, double drs,
                            int nr, int off, double* x_int, double* x_half);
void launch_coefficients(cudaStream_t st, int prec, double M, double a, int s, int m,
                         double rstar_min, double drs, double dth, double dt, int nr, int nth,
                         int pitch, const double* x_int, const double* x_half, void* coef_h,
                         void* coef_i);
void launch_tables_1d(cudaStream_t st, double M, double a, int s, int m, double drs, double dth,
                      double dt, int nr, int nth, const double* x_int, const double* x_half,
                      RTab2* rtab, ThTab* thtab);
void launch_profile(cudaStream_t st, double M, double a, double rstar_min, double drs, int off,
                    double dth, double rs0, double sig_r, double sig_t, double drs0_dr0,
                    const double* x_int, const double* x_half, const SourceDev& src, int prec);
// moving particle: the prefactor profile Q on the window and the per-step tables of
// src (traj: device copy of the samples, [n_samples][4])
void launch_trajectory(cudaStream_t st, double M, double a, int m, double rstar_min, double drs,
                       int off, double dth, double sig_r, double sig_t, const double* x_int,
                       const double* x_half, const double* traj, int64_t n_samples,
                       const SourceDev& src, int prec);
// teuk_step.cu
cudaError_t prepare_step_kernels();
int step_resident_blocks(int prec, int threads);  // blocks of the step kernel the GPU holds at once
// part (device, may be null): block b covers the columns [part[b], part[b+1]) of a
// partition into ceil((n_rstar - 2) / strip) pieces, instead of uniform strips
void launch_step(cudaStream_t st, const InstDev& d, int64_t step, int bin, int strip,
                 const int* part = nullptr);
void launch_extract(cudaStream_t st, const InstDev& d, int64_t step, int bin);
// *base += k (one thread): closes a replayed graph of k per-step launches
void launch_advance_step(cudaStream_t st, int64_t* base, int64_t k);
// moving: some instance of the class has a moving particle (selects the kernel that
// carries the per-step Gaussian tables)
void launch_batched_step(cudaStream_t st, int prec, const BatchDev& b, int grid, int threads,
                         bool moving);
int batched_grid(int prec, int threads);
void launch_batched_extract(cudaStream_t st, int prec, const BatchDev& b, int max_nth);
// teuk_resident.cu: whether (and how) an instance fits the resident kernel with halo h
// (all blocks resident at once, one block per run of columns, aiming at bps blocks per
// SM: with several, one block's halo wait overlaps another's arithmetic), and its launch
bool resident_plan(int prec, int nr, int pitch, int h, int bps, ResidentPlan* plan);
// cooperative: one launch for a whole teuk_step_n (blocks wait on one another); otherwise a
// blocked launch of at most h steps (a.no_wait), issued with programmatic dependent launch
cudaError_t launch_resident(cudaStream_t st, const ResidentArgs& a, const ResidentPlan& plan,
                            bool cooperative = true);
// teuk_aux.cu
void launch_import_state(cudaStream_t st, const InstDev& d, int bin, const double* u);
void launch_export_state(cudaStream_t st, const InstDev& d, int bin, double* u);
void launch_scan_finite(cudaStream_t st, const InstDev& d, int bin);
void launch_wave_sum(cudaStream_t st, const double2* wave, int64_t cap, int nth, double dth,
                     int64_t level0, int64_t k_count, double2* out);
// teuk_adjoint.cu
// Co-state of one time level (teuk_adjoint.cu): F and P planes ([nr][pitch] complex,
// double2 for FP64 instances, float2 otherwise) and, for FP32, their compensation
// planes (float2; the value is v - c).
struct CoLevel { void* F; void* P; void* Fc; void* Pc; };
// lam = E^T gbar: the co-state that starts the reverse sweep
void launch_adj_init(cudaStream_t st, const InstDev& d, const double2* gbar, const CoLevel& out);
// the fused reverse step (lam^n from lam^{n+1}): strip length and block count from
// adj_step_plan; wh, wi (null without a source): the step's ring slot of the window
// co-states, mu_Pi at the half-node window ([nj][nh]) and lam'_Pi at the integer-node
// window ([nj][ni]), complex in the co-state's type
int adj_step_plan(const InstDev& d, int* strip);
void launch_adj_step(cudaStream_t st, const InstDev& d, const CoLevel& lin, const double2* gbar,
                     const CoLevel& lout, int strip, void* wh, void* wi);
// bytes of one ring slot (the half-node window, then the integer-node window)
size_t adj_window_bytes(const InstDev& d);
// source gradients gA[k], gR[k] of the steps k0 .. k0 + count - 1 of a sweep starting at
// step0, from ring slots k % slots
void launch_adj_src_grad(cudaStream_t st, const InstDev& d, int64_t step0, int64_t k0, int64_t count,
                         int slots, const void* ring, double* gA, double* gR);
// built-in loss of records level0 .. level0 + count - 1 (ring wave of cap slots):
// lossrec[0 .. count), their cotangents into slots (g0 + k) % gcap of gbar
void launch_loss_records(cudaStream_t st, const double2* wave, int64_t cap, int nth,
                         int64_t level0, int64_t count, double r6, double* lossrec,
                         double2* gbar, int64_t gcap, int64_t g0);
void launch_ordered_sum(cudaStream_t st, const double* v, int64_t n, double* out);

}  // namespace teuk
