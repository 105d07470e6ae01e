// teuk_adjoint.cu -- transpose of one Lax-Wendroff step (Eqs. 13-14), as gathers.
//
// The step is affine and complex-linear in u:  u^{n+1} = P (u^n + C(H u^n)) + A_n s_n,
// with H the predictor of Eq. (13) (integer nodes -> half nodes), C the corrector
// increment of Eq. (14) (half nodes -> integer nodes) and P the radial boundary
// condition (zero at i = 0 and i = n_rstar - 1).  With the real inner product
// <x, y> = sum Re(conj(x) y), the transpose of y += c x is x += conj(c) y.  So one
// reverse step is
//   lam'  = P lam^{n+1}
//   mu    = C^T lam'                       (half nodes)
//   lam^n = lam' + H^T mu + E^T gbar_n     (integer nodes), all in one reverse-step kernel
// and the source enters the gradients as
//   dL/dA_n  = <mu_Pi, (dt/2) e_p P_half> + <lam'_Pi, dt e_c P_int>
//   dL/dr0  += A_n (<mu_Pi, (dt/2) d(e_p P_half)/dr0> + <lam'_Pi, dt d(e_c P_int)/dr0>)
// with e_p = e^{-i(omega t_n + phase0)}, e_c the same at t_n + dt/2 (the step stores
// mu_Pi and lam'_Pi over the source window; adj_src_grad_kernel forms the sums).
// Coefficients (g, E1, E2, ep, em, E3, scaled as in teuk_setup.cu) are read from the 2D
// tables for FP64 and double-float instances and formed from the 1D tables, as the
// forward kernels form them, for FP32 instances; in
// the corrector's angular term  ep Phi~(j+1) + em Phi~(j-1) + (E3 - ep - em) Phi~(j)
// the ghost rows fold back onto rows 0 and n_theta-1 with the sign of the pole
// condition.  The co-state lam and mu are FP64 for FP64 instances; for FP32 instances
// they are FP32, lam compensated like the forward state (value hi - c, each step's
// increment added with Kahan's compensated sum), the gradient sums FP64 either way.
#include <type_traits>

#include "teuk_df.cuh"
#include "teuk_internal.cuh"
#include "teuk_step_common.cuh"

namespace teuk {

template <typename R>
struct Z { R x, y; };
template <typename R>
__device__ __forceinline__ Z<R> zadd(Z<R> a, Z<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ Z<R> zscale(R s, Z<R> a) { return {s * a.x, s * a.y}; }
// conj(cr + i ci) * z
template <typename R>
__device__ __forceinline__ Z<R> zconjmul(R cr, R ci, Z<R> z) {
    return {cr * z.x + ci * z.y, cr * z.y - ci * z.x};
}

template <typename R> struct R2T;
template <> struct R2T<double> { using V = double2; };
template <> struct R2T<float> { using V = float2; };

// One co-state plane (complex, [nr][pitch]) and, for FP32, its compensation plane.
template <typename R>
struct CoPlane {
    typename R2T<R>::V* v;
    float2* c;   // FP32 only: value = v - c
    __device__ __forceinline__ Z<R> ld(size_t o) const {
        const typename R2T<R>::V a = v[o];
        if constexpr (sizeof(R) == 4) {
            const float2 b = c[o];
            return {a.x - b.x, a.y - b.y};
        } else {
            return {a.x, a.y};
        }
    }
};
template <typename R>
__device__ __forceinline__ CoPlane<R> coplane(const CoLevel& L, int k) {
    return {(typename R2T<R>::V*)(k == 0 ? L.F : L.P), (float2*)(k == 0 ? L.Fc : L.Pc)};
}
template <typename R>
__device__ __forceinline__ Z<R> ldv(const void* p, size_t o) {
    const typename R2T<R>::V a = ((const typename R2T<R>::V*)p)[o];
    return {a.x, a.y};
}
template <typename R>
__device__ __forceinline__ void stv(void* p, size_t o, Z<R> z) {
    ((typename R2T<R>::V*)p)[o] = {z.x, z.y};
}
template <typename R>
__device__ __forceinline__ Z<R> gld(const double2* p, size_t o) {
    const double2 a = p[o];
    return {(R)a.x, (R)a.y};
}

template <typename T, typename R>
__device__ __forceinline__ R cget(const T* tab, size_t pl, int k, size_t o) {
    if constexpr (std::is_same<T, DF>::value) return (R)tab[(size_t)k * pl + o].to_double();
    else return (R)tab[(size_t)k * pl + o];
}

// Compensated add of an increment to one co-state node (FP32): value = v - c.
__device__ __forceinline__ void kahan_node(float2& v, float2& c, Z<float> dlt) {
    float yx = __fsub_rn(dlt.x, c.x), yy = __fsub_rn(dlt.y, c.y);
    float tx = __fadd_rn(v.x, yx), ty = __fadd_rn(v.y, yy);
    c.x = __fsub_rn(__fsub_rn(tx, v.x), yx);
    c.y = __fsub_rn(__fsub_rn(ty, v.y), yy);
    v.x = tx;
    v.y = ty;
}

// lam = E^T gbar (the start of the reverse sweep).
template <typename R>
__global__ void adj_init_kernel(InstDev d, const double2* gbar, CoLevel out) {
    int j = blockIdx.y * blockDim.x + threadIdx.x;   // theta row
    int i = blockIdx.x;                              // r* column
    if (j >= d.pitch || i >= d.nr) return;
    size_t o = node_index(d, i, j);
    Z<double> a = {0, 0};
    if (gbar && i == d.i_e) a = zscale(1.0 - d.f_e, gld<double>(gbar, j));
    if (gbar && i == d.i_e + 1) a = zscale(d.f_e, gld<double>(gbar, j));
    stv<R>(out.F, o, Z<R>{(R)a.x, (R)a.y});
    stv<R>(out.P, o, Z<R>{0, 0});
    if constexpr (sizeof(R) == 4) {
        ((float2*)out.Fc)[o] = make_float2(0.f, 0.f);
        ((float2*)out.Pc)[o] = make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------ fused reverse step
// One reverse step in one pass over the grid: lam^n = P lam^{n+1} + H^T (C^T P lam^{n+1})
// + E^T gbar.  A block holds one theta column (one thread a row) and streams along r*
// over a strip of output columns [c0, c1): at half node h it forms mu(h) = C^T lam' from
// the integer columns h and h+1 (the angular neighbours of lam'_Pi through shared
// memory), then lam^n(h) = H^T mu from the half nodes h-1 and h (the angular neighbours
// of mu_Pi through shared memory), so neither mu nor lam' is written to memory.  The
// arithmetic of each node is that of the two gather passes in the same order
// (corrector: integer node h, then h+1; predictor: half node h-1, then h).  Over the
// source window the step also stores mu_Pi (half nodes) and lam'_Pi (integer nodes) into
// one slot of a ring, from which adj_src_grad_kernel forms the source gradients of many
// steps at once, off the step's critical path.

// theta_cotangent with the angular neighbours given: lm, l0, lp the Pi cotangents of
// rows j-1, j, j+1 of column node o.
template <typename T, typename R>
__device__ __forceinline__ Z<R> theta_cot3(const T* tab, size_t pl, size_t o, int j, int nth, Z<R> lm,
                                           Z<R> l0, Z<R> lp, R g) {
    R ep0 = cget<T, R>(tab, pl, C_EP, o), em0 = cget<T, R>(tab, pl, C_EM, o);
    Z<R> r = zconjmul(cget<T, R>(tab, pl, C_E3R, o) - ep0 - em0, cget<T, R>(tab, pl, C_E3I, o), l0);
    if (j >= 1) r = zadd(r, zscale(cget<T, R>(tab, pl, C_EP, o - 1), lm));
    else r = zadd(r, zscale(g * em0, l0));
    if (j + 1 < nth) r = zadd(r, zscale(cget<T, R>(tab, pl, C_EM, o + 1), lp));
    else r = zadd(r, zscale(g * ep0, l0));
    return r;
}

// The co-state of one node as stored: FP64 value, or FP32 (v, c) pairs with value v - c.
template <typename R>
struct CoNode {
    Z<R> F, P;          // values
    float2 vF, cF, vP, cP;   // FP32: the stored pairs
};
template <typename R>
__device__ __forceinline__ CoNode<R> co_load(const CoLevel& L, size_t o) {
    CoNode<R> n{};
    if constexpr (sizeof(R) == 4) {
        n.vF = ((const float2*)L.F)[o];
        n.cF = ((const float2*)L.Fc)[o];
        n.vP = ((const float2*)L.P)[o];
        n.cP = ((const float2*)L.Pc)[o];
        n.F = {n.vF.x - n.cF.x, n.vF.y - n.cF.y};
        n.P = {n.vP.x - n.cP.x, n.vP.y - n.cP.y};
    } else {
        n.F = ldv<R>(L.F, o);
        n.P = ldv<R>(L.P, o);
    }
    return n;
}

// Source gradients of step n.  With e = e^{-i phi} the phase of a sub-step and
// de = d e / d r0,
//   dL/dA_n  = Re( (dt/2) e_p S_h + dt e_c S_i ),
//   dL/dr0  += A_n Re( (dt/2) (de_p S_h + e_p S'_h) + dt (de_c S_i + e_c S'_i) ),
// where S_h = sum conj(mu_Pi) P_half and S'_h = sum conj(mu_Pi) dP_half over the
// half-node window, S_i and S'_i the same with lam'_Pi over the integer-node window
// (zero off the interior columns).  One block a step: the steps k0 .. k0 + count - 1 of
// a sweep (absolute step step0 + k); ring slot k % slots holds the step's half-node
// window ([nj][nh]) followed by its integer-node window ([nj][ni]).  Each
// thread sums its nodes (t, t + blockDim, ...) in FP64, the threads are added in a fixed
// tree, so the result does not depend on the scheduling.
constexpr int kSrcGradThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kSrcGradThreads) adj_src_grad_kernel(InstDev d, int64_t step0, int64_t k0,
                                                                       int slots, const void* ring,
                                                                       double* gA, double* gR) {
    using V = typename R2T<R>::V;
    const SourceDev& s = d.src;
    const int64_t k = k0 + blockIdx.x, n = step0 + k;
    const size_t nhw = (size_t)s.nh * s.nj, niw = (size_t)s.ni * s.nj;
    const V* Hw = (const V*)ring + (size_t)(k % slots) * (nhw + niw);
    const V* Iw = Hw + nhw;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // S_h, S'_h, S_i, S'_i (re, im)
    for (size_t q = threadIdx.x; q < nhw; q += blockDim.x) {
        const V m = Hw[q];
        const double lx = (double)m.x, ly = (double)m.y;
        const double2 P = s.P_half[q], dP = s.dP_half[q];
        acc[0] += lx * P.x + ly * P.y;
        acc[1] += lx * P.y - ly * P.x;
        acc[2] += lx * dP.x + ly * dP.y;
        acc[3] += lx * dP.y - ly * dP.x;
    }
    for (size_t q = threadIdx.x; q < niw; q += blockDim.x) {
        const V m = Iw[q];
        const double lx = (double)m.x, ly = (double)m.y;
        const double2 P = s.P_int[q], dP = s.dP_int[q];
        acc[4] += lx * P.x + ly * P.y;
        acc[5] += lx * P.y - ly * P.x;
        acc[6] += lx * dP.x + ly * dP.y;
        acc[7] += lx * dP.y - ly * dP.x;
    }
    __shared__ double wred[kSrcGradThreads / 32][8];
    __shared__ double S[8];
    __shared__ Z<double> ph[4];   // e_p, e_c, de_p, de_c
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double x = acc[v];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) wred[warp][v] = x;
    }
    __syncthreads();
    if (t < 8) {
        double x = 0.0;
        for (int w = 0; w < kSrcGradThreads / 32; ++w) x += wred[w][t];
        S[t] = x;
    }
    if (t == 64 || t == 96) {   // the two sub-step phases, on two other warps
        const double tt = (double)n * d.dt + (t == 64 ? 0.0 : 0.5 * d.dt);
        double sn, cs;
        sincos(s.omega * tt + s.phase0, &sn, &cs);
        const double kk = tt * s.domega + s.dphase0;   // e = (cos, -sin); de = -i k e
        const Z<double> e = {cs, -sn};
        ph[t == 64 ? 0 : 1] = e;
        ph[t == 64 ? 2 : 3] = Z<double>{kk * e.y, -kk * e.x};
    }
    __syncthreads();
    if (t != 0) return;
    const double A = (s.amps != nullptr && n < s.n_amps) ? s.amps[n] : 1.0;
    auto re_mul = [](Z<double> a, double bx, double by) { return a.x * bx - a.y * by; };
    const double hd = 0.5 * d.dt;
    gA[k] = hd * re_mul(ph[0], S[0], S[1]) + d.dt * re_mul(ph[1], S[4], S[5]);
    gR[k] = A * (hd * (re_mul(ph[2], S[0], S[1]) + re_mul(ph[0], S[2], S[3])) +
                 d.dt * (re_mul(ph[3], S[4], S[5]) + re_mul(ph[1], S[6], S[7])));
}

// Programmatic dependent launch of consecutive reverse steps: a block releases the next
// step's launch on entry; the next step's blocks set up what depends only on constant
// data and wait (griddepcontrol.wait: the previous grid has completed and its writes are
// visible) before they read the co-state or write anything to global memory.
__device__ __forceinline__ void adj_release_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void adj_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// kMaxT: the largest block this instance serves (256: columns of up to 256 rows, with
// the register budget of several blocks per SM; 512: up to 512 rows, one block per SM;
// 1024: taller columns)
template <typename T, typename R, int kMaxT>
__global__ void __launch_bounds__(kMaxT) adj_step_kernel(InstDev d, CoLevel lin, const double2* gbar,
                                                         CoLevel lout, int strip, void* wh, void* wi) {
    extern __shared__ __align__(16) unsigned char adj_smem[];
    adj_release_next();
    Z<R>* LB = (Z<R>*)adj_smem;                 // [2][pitch] lam'_Pi of a column
    Z<R>* MB = LB + 2 * (size_t)d.pitch;        // [2][pitch] mu_Pi of a half node
    const int j = threadIdx.x, nth = d.nth, nr = d.nr, pitch = d.pitch;
    const bool row_ok = j < nth;
    const int c0 = blockIdx.x * strip, c1 = min(nr, c0 + strip);   // output columns [c0, c1)
    const T* ci = (const T*)d.coef_i;
    const T* ch = (const T*)d.coef_h;
    const size_t pl = plane_elems(d);
    const R g = (R)d.ghost, hdt = (R)(0.5 * d.dt);
    constexpr bool kComp = sizeof(R) == 4;
    const SourceDev& s = d.src;
    // wh, wi: this step's ring slot of the window co-states (null: no source)
    // lam' = P lam^{n+1} at column col (zero at the boundary columns and outside)
    auto lam_at = [&](int col) {
        CoNode<R> z{};
        if (row_ok && col >= 1 && col <= nr - 2) z = co_load<R>(lin, node_index(d, col, j));
        return z;
    };
    auto nb3 = [&](const Z<R>* buf, int sl, Z<R>& lm, Z<R>& lp) {
        const Z<R>* b = buf + (size_t)sl * pitch;
        lm = j >= 1 ? b[j - 1] : Z<R>{0, 0};
        lp = j + 1 < nth ? b[j + 1] : Z<R>{0, 0};
    };
    adj_wait_prev();
    CoNode<R> l_cur = lam_at(c0 - 1), l_next;
    LB[(size_t)((c0 - 1) & 1) * pitch + j] = l_cur.P;
    Z<R> mu_prevF = {0, 0}, mu_prevP = {0, 0};
    for (int h = c0 - 1; h <= c1 - 1; ++h) {
        // A: lam' of column h+1
        l_next = lam_at(h + 1);
        LB[(size_t)((h + 1) & 1) * pitch + j] = l_next.P;
        __syncthreads();
        // C: mu at half node h = C^T lam' from the integer columns h (right neighbour of
        // this half node, sign +1) and h+1 (left neighbour, sign -1)
        Z<R> muF = {0, 0}, muP = {0, 0};
        if (row_ok && h >= 0 && h <= nr - 2) {
            for (int side = 0; side < 2; ++side) {
                const int col = h + side;
                if (col < 1 || col > nr - 2) continue;
                const R sR = side == 0 ? R(1) : R(-1);
                const size_t o = node_index(d, col, j);
                const CoNode<R>& L = side == 0 ? l_cur : l_next;
                Z<R> lm, lp;
                nb3(LB, col & 1, lm, lp);
                const R G = cget<T, R>(ci, pl, C_G, o);
                const Z<R> tc = theta_cot3<T, R>(ci, pl, o, j, nth, lm, L.P, lp, g);
                muF = zadd(muF, zscale(-sR * G, L.F));
                muF = zadd(muF, zscale(sR, zconjmul(cget<T, R>(ci, pl, C_E2R, o), cget<T, R>(ci, pl, C_E2I, o), L.P)));
                muF = zadd(muF, zscale(R(0.5), tc));
                muP = zadd(muP, zscale((R)(0.5 * d.dt), L.F));
                muP = zadd(muP, zscale(sR * G, L.P));
                muP = zadd(muP, zscale(R(0.5), zconjmul(cget<T, R>(ci, pl, C_E1R, o), cget<T, R>(ci, pl, C_E1I, o), L.P)));
            }
            if (wh && h >= c0) {   // half-node window: mu_Pi (half node c0 - 1 is the
                                   // previous block's)
                const int a = h - s.h_lo, bb = j - s.j_lo;
                if ((unsigned)a < (unsigned)s.nh && (unsigned)bb < (unsigned)s.nj)
                    stv<R>(wh, (size_t)bb * s.nh + a, muP);
            }
        }
        MB[(size_t)(h & 1) * pitch + j] = muP;
        __syncthreads();
        // F: lam^n at integer column h from the half nodes h-1 (this column is their right
        // input, sign +1) and h (left input, sign -1)
        if (h >= c0 && row_ok) {
            const int i = h;
            const size_t o = node_index(d, i, j);
            const bool interior = i >= 1 && i <= nr - 2;
            Z<R> aF = {0, 0}, aP = {0, 0};
            if constexpr (!kComp) {
                if (interior) {
                    aF = l_cur.F;
                    aP = l_cur.P;
                }
            }
            for (int side = 0; side < 2; ++side) {
                const int hh = i - 1 + side;
                if (hh < 0 || hh > nr - 2) continue;
                const R sR = side == 0 ? R(1) : R(-1);
                const size_t oh = node_index(d, hh, j);
                const Z<R> MF = side == 0 ? mu_prevF : muF, MP = side == 0 ? mu_prevP : muP;
                Z<R> mm, mp;
                nb3(MB, hh & 1, mm, mp);
                const R G = cget<T, R>(ch, pl, C_G, oh);
                const Z<R> tc = theta_cot3<T, R>(ch, pl, oh, j, nth, mm, MP, mp, g);
                aF = zadd(aF, zscale(R(0.5) - sR * G, MF));
                aF = zadd(aF, zscale(sR, zconjmul(cget<T, R>(ch, pl, C_E2R, oh), cget<T, R>(ch, pl, C_E2I, oh), MP)));
                aF = zadd(aF, zscale(R(0.5), tc));
                aP = zadd(aP, zscale(R(0.5) * hdt, MF));
                aP = zadd(aP, zscale(R(0.5) + sR * G, MP));
                aP = zadd(aP, zscale(R(0.5), zconjmul(cget<T, R>(ch, pl, C_E1R, oh), cget<T, R>(ch, pl, C_E1I, oh), MP)));
            }
            if (gbar) {   // transpose of the linear extraction between i_e and i_e + 1
                if (i == d.i_e) aF = zadd(aF, zscale((R)(1.0 - d.f_e), gld<R>(gbar, j)));
                if (i == d.i_e + 1) aF = zadd(aF, zscale((R)d.f_e, gld<R>(gbar, j)));
            }
            if constexpr (kComp) {
                float2 vF = {0.f, 0.f}, cF = {0.f, 0.f}, vP = {0.f, 0.f}, cP = {0.f, 0.f};
                if (interior) {
                    vF = l_cur.vF;
                    cF = l_cur.cF;
                    vP = l_cur.vP;
                    cP = l_cur.cP;
                }
                kahan_node(vF, cF, aF);
                kahan_node(vP, cP, aP);
                if (TK_IN(d.status, o, pl)) {
                    ((float2*)lout.F)[o] = vF;
                    ((float2*)lout.Fc)[o] = cF;
                    ((float2*)lout.P)[o] = vP;
                    ((float2*)lout.Pc)[o] = cP;
                }
            } else if (TK_IN(d.status, o, pl)) {
                stv<R>(lout.F, o, aF);
                stv<R>(lout.P, o, aP);
            }
            if (wi) {   // integer-node window: lam'_Pi (zero off the interior columns)
                const int a = i - s.i_lo, bb = j - s.j_lo;
                if ((unsigned)a < (unsigned)s.ni && (unsigned)bb < (unsigned)s.nj)
                    stv<R>(wi, (size_t)bb * s.ni + a, interior ? l_cur.P : Z<R>{0, 0});
            }
        }
        l_cur = l_next;
        mu_prevF = muF;
        mu_prevP = muP;
    }
}

// The FP32 co-state (FP32 and FP32-Kahan instances): the same reverse step with the
// coefficients formed in registers from the 1D tables (form_coefs2, the split angular
// form turned back into ep = A + B, em = A - B), i.e. the coefficients the forward FP32
// kernels compute, instead of 2D tables: the reverse step is then the transpose of the
// forward operator as it is evaluated, and it reads no coefficient tables.  Each column's
// coefficients are formed once per step and used at once for both nodes they enter: the
// corrector coefficients of column c enter mu(c-1) (as its right node) and mu(c) (as its
// left node), those of half node c enter lam(c) and lam(c+1); the partial sums are
// carried to the next column, so every sum is formed in the order of the gather form
// (left neighbour first).
struct CfF { float g, e1r, e1i, e2r, e2i, ep, em, e3r, e3i; };

__device__ __forceinline__ Z<float> theta_cot_v(const CfF& c, float ep_m, float em_p, Z<float> lm,
                                                Z<float> l0, Z<float> lp, int j, int nth, float g) {
    Z<float> r = zconjmul(c.e3r - c.ep - c.em, c.e3i, l0);
    if (j >= 1) r = zadd(r, zscale(ep_m, lm));
    else r = zadd(r, zscale(g * c.em, l0));
    if (j + 1 < nth) r = zadd(r, zscale(em_p, lp));
    else r = zadd(r, zscale(g * c.ep, l0));
    return r;
}

// columns of radial tables the FP32 reverse step stages in shared memory (strips of up
// to kAdjRtCols - 2 columns; longer strips read the tables from global memory)
constexpr int kAdjRtCols = 64;

template <int kMaxT>
__global__ void __launch_bounds__(kMaxT) adj_step_kernel_f32(InstDev d, CoLevel lin, const double2* gbar,
                                                             CoLevel lout, int strip, void* wh, void* wi) {
    using R = float;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    adj_release_next();
    const int j = threadIdx.x, nth = d.nth, nr = d.nr, pitch = d.pitch;
    Z<R>* LB = (Z<R>*)adj_smem;                   // [2][pitch] lam'_Pi of a column
    Z<R>* MB = LB + 2 * (size_t)pitch;            // [2][pitch] mu_Pi of a half node
    float4* EB = (float4*)(MB + 2 * (size_t)pitch);   // [3][pitch] {ep, em} of node, half node
    RTab2* RT = (RTab2*)(EB + 3 * (size_t)pitch);      // radial tables of columns c0-1 .. c1
    const bool row_ok = j < nth;
    const int c0 = blockIdx.x * strip, c1 = min(nr, c0 + strip);   // output columns [c0, c1)
    const bool rt_smem = strip + 2 <= kAdjRtCols;   // else the tables are read from global
    const R g = (R)d.ghost, hdt = (R)(0.5 * d.dt), qdt = (R)(0.5 * d.dt);
    const SourceDev& s = d.src;
    // wh, wi: this step's ring slot of the window co-states (null: no source)
    RowTab<PK> rt;
    rt.load(d.thtab, j, row_ok);
    auto lam_at = [&](int col) {
        CoNode<R> z{};
        if (row_ok && col >= 1 && col <= nr - 2) z = co_load<R>(lin, node_index(d, col, j));
        return z;
    };
    // the stored pairs of a column, loaded one column ahead of use (zero outside the
    // interior columns, as lam_at); as_node forms the values when the column is used
    struct CoRaw { float2 vF, cF, vP, cP; };
    auto raw_at = [&](int col) {
        CoRaw z{};
        if (row_ok && col >= 1 && col <= nr - 2) {
            const size_t o = node_index(d, col, j);
            z.vF = __ldg((const float2*)lin.F + o);
            z.cF = __ldg((const float2*)lin.Fc + o);
            z.vP = __ldg((const float2*)lin.P + o);
            z.cP = __ldg((const float2*)lin.Pc + o);
        }
        return z;
    };
    auto as_node = [](const CoRaw& r) {
        CoNode<R> n;
        n.vF = r.vF;
        n.cF = r.cF;
        n.vP = r.vP;
        n.cP = r.cP;
        n.F = {r.vF.x - r.cF.x, r.vF.y - r.cF.y};
        n.P = {r.vP.x - r.cP.x, r.vP.y - r.cP.y};
        return n;
    };
    // coefficients of column col: node col (ci) and half node col+1/2 (ch)
    auto form = [&](int col, CfF& ci, CfF& ch) {
        float2 cf2[kNCoef];
        if (col >= 0 && col <= nr - 1) {
            form_coefs2(rt_smem ? RT[col - (c0 - 1)] : d.rtab[col], rt.t, cf2);
        } else {
#pragma unroll
            for (int q = 0; q < kNCoef; ++q) cf2[q] = make_float2(0.f, 0.f);
        }
        auto pick = [&](bool half) {
            auto v = [&](int q) { return half ? cf2[q].x : cf2[q].y; };
            return CfF{v(C_G), v(C_E1R), v(C_E1I), v(C_E2R), v(C_E2I), __fadd_rn(v(C_EP), v(C_EM)),
                       __fsub_rn(v(C_EP), v(C_EM)), v(C_E3R), v(C_E3I)};
        };
        ci = pick(false);
        ch = pick(true);
    };
    auto nb3 = [&](const Z<R>* buf, int sl, Z<R>& lm, Z<R>& lp) {
        const Z<R>* b = buf + (size_t)sl * pitch;
        lm = j >= 1 ? b[j - 1] : Z<R>{0, 0};
        lp = j + 1 < nth ? b[j + 1] : Z<R>{0, 0};
    };
    // corrector contribution of node col (coefficients c, co-state L) to a half node on
    // its right (sR = +1) or left (sR = -1)
    auto e3 = [](int col) { return (col + 3) % 3; };   // EB slot of column col >= -1
    auto corr = [&](const CfF& c, const CoNode<R>& L, int col, R sR, Z<R>& muF, Z<R>& muP) {
        const int sl = col & 1;
        Z<R> lm, lp;
        nb3(LB, sl, lm, lp);
        const float4 em = EB[(size_t)e3(col) * pitch + (j >= 1 ? j - 1 : j)];   // row j-1
        const float4 ep = EB[(size_t)e3(col) * pitch + (j + 1 < nth ? j + 1 : j)];   // row j+1
        const Z<R> tc = theta_cot_v(c, em.x, ep.y, lm, L.P, lp, j, nth, g);
        muF = zadd(muF, zscale(-sR * c.g, L.F));
        muF = zadd(muF, zscale(sR, zconjmul(c.e2r, c.e2i, L.P)));
        muF = zadd(muF, zscale(R(0.5), tc));
        muP = zadd(muP, zscale(hdt, L.F));
        muP = zadd(muP, zscale(sR * c.g, L.P));
        muP = zadd(muP, zscale(R(0.5), zconjmul(c.e1r, c.e1i, L.P)));
    };
    // predictor contribution of half node hh (coefficients c, cotangent MF, MP) to the node
    // on its right (sR = +1) or left (sR = -1)
    auto pred = [&](const CfF& c, Z<R> MF, Z<R> MP, int hh, R sR, Z<R>& aF, Z<R>& aP) {
        const int sl = hh & 1;
        Z<R> mm, mp;
        nb3(MB, sl, mm, mp);
        const float4 em = EB[(size_t)e3(hh) * pitch + (j >= 1 ? j - 1 : j)];   // row j-1
        const float4 ep = EB[(size_t)e3(hh) * pitch + (j + 1 < nth ? j + 1 : j)];   // row j+1
        const Z<R> tc = theta_cot_v(c, em.z, ep.w, mm, MP, mp, j, nth, g);
        aF = zadd(aF, zscale(R(0.5) - sR * c.g, MF));
        aF = zadd(aF, zscale(sR, zconjmul(c.e2r, c.e2i, MP)));
        aF = zadd(aF, zscale(R(0.5), tc));
        aP = zadd(aP, zscale(R(0.5) * qdt, MF));
        aP = zadd(aP, zscale(R(0.5) + sR * c.g, MP));
        aP = zadd(aP, zscale(R(0.5), zconjmul(c.e1r, c.e1i, MP)));
    };
    // the strip's radial tables into shared memory (one broadcast read per column later)
    if (rt_smem) {
        const int ncols = c1 - c0 + 2;
        for (int q = threadIdx.x; q < ncols * 8; q += blockDim.x) {
            const int k = q >> 3, col = c0 - 1 + k;
            if (col >= 0 && col <= nr - 1) ((float4*)(RT + k))[q & 7] = __ldg((const float4*)(d.rtab + col) + (q & 7));
        }
        __syncthreads();
    }
    adj_wait_prev();
    // prologue: column c0 - 1
    CoNode<R> l_cur = lam_at(c0 - 1);
    CfF ci_cur, ch_cur;
    form(c0 - 1, ci_cur, ch_cur);
    LB[(size_t)((c0 - 1) & 1) * pitch + j] = l_cur.P;
    EB[(size_t)e3(c0 - 1) * pitch + j] = make_float4(ci_cur.ep, ci_cur.em, ch_cur.ep, ch_cur.em);
    __syncthreads();
    Z<R> muF_part = {0, 0}, muP_part = {0, 0};      // mu(h): the left node's share
    if (row_ok && c0 - 1 >= 1 && c0 - 1 <= nr - 2) corr(ci_cur, l_cur, c0 - 1, R(1), muF_part, muP_part);
    Z<R> aF_part = {0, 0}, aP_part = {0, 0};        // lam(h): the left half node's share
    CoRaw r_next = raw_at(c0);
    for (int h = c0 - 1; h <= c1 - 1; ++h) {
        // A: column h+1: its co-state (loaded one column ahead) and coefficients
        const CoNode<R> l_next = as_node(r_next);
        r_next = raw_at(h + 2);
        CfF ci_n, ch_n;
        form(h + 1, ci_n, ch_n);
        LB[(size_t)((h + 1) & 1) * pitch + j] = l_next.P;
        EB[(size_t)e3(h + 1) * pitch + j] = make_float4(ci_n.ep, ci_n.em, ch_n.ep, ch_n.em);
        __syncthreads();
        // C: mu(h) = its left node's share + the right node h+1; the left share of mu(h+1)
        Z<R> muF = muF_part, muP = muP_part, mfn = {0, 0}, mpn = {0, 0};
        const bool half_ok = h >= 0 && h <= nr - 2;
        if (row_ok && h + 1 >= 1 && h + 1 <= nr - 2) {
            if (half_ok) corr(ci_n, l_next, h + 1, R(-1), muF, muP);
            if (h + 1 <= nr - 2) corr(ci_n, l_next, h + 1, R(1), mfn, mpn);
        }
        if (!half_ok || !row_ok) muF = muP = Z<R>{0, 0};
        if (wh && half_ok && row_ok && h >= c0) {
            const int a = h - s.h_lo, bb = j - s.j_lo;
            if ((unsigned)a < (unsigned)s.nh && (unsigned)bb < (unsigned)s.nj)
                stv<R>(wh, (size_t)bb * s.nh + a, muP);
        }
        MB[(size_t)(h & 1) * pitch + j] = muP;
        __syncthreads();
        // F: half node h's shares of lam(h) (completing it) and lam(h+1)
        Z<R> aF = aF_part, aP = aP_part, afn = {0, 0}, apn = {0, 0};
        if (row_ok && half_ok) {
            pred(ch_cur, muF, muP, h, R(-1), aF, aP);
            pred(ch_cur, muF, muP, h, R(1), afn, apn);
        }
        if (h >= c0 && row_ok) {
            const int i = h;
            const size_t o = node_index(d, i, j);
            const bool interior = i >= 1 && i <= nr - 2;
            if (gbar) {
                if (i == d.i_e) aF = zadd(aF, zscale((R)(1.0 - d.f_e), gld<R>(gbar, j)));
                if (i == d.i_e + 1) aF = zadd(aF, zscale((R)d.f_e, gld<R>(gbar, j)));
            }
            float2 vF = {0.f, 0.f}, cF = {0.f, 0.f}, vP = {0.f, 0.f}, cP = {0.f, 0.f};
            if (interior) {
                vF = l_cur.vF;
                cF = l_cur.cF;
                vP = l_cur.vP;
                cP = l_cur.cP;
            }
            kahan_node(vF, cF, aF);
            kahan_node(vP, cP, aP);
            if (TK_IN(d.status, o, plane_elems(d))) {
                ((float2*)lout.F)[o] = vF;
                ((float2*)lout.Fc)[o] = cF;
                ((float2*)lout.P)[o] = vP;
                ((float2*)lout.Pc)[o] = cP;
            }
            if (wi) {
                const int a = i - s.i_lo, bb = j - s.j_lo;
                if ((unsigned)a < (unsigned)s.ni && (unsigned)bb < (unsigned)s.nj)
                    stv<R>(wi, (size_t)bb * s.ni + a, interior ? l_cur.P : Z<R>{0, 0});
            }
        }
        l_cur = l_next;
        ch_cur = ch_n;
        muF_part = mfn;
        muP_part = mpn;
        aF_part = afn;
        aP_part = apn;
    }
}

// Loss of the built-in |r_ext^3 W|^2: per record, lossrec[k] = r^6 sum_j |W_k[j]|^2 (j
// ascending) and gbar_k = 2 r^6 W_k.  Records are read from a ring (slot level % cap),
// gbar_k is written to slot (g0 + k) % gcap of another.
__global__ void loss_records_kernel(const double2* wave, int64_t cap, int nth, int64_t level0,
                                    int64_t count, double r6, double* lossrec, double2* gbar,
                                    int64_t gcap, int64_t g0) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    const double2* w = wave + (size_t)((level0 + k) % cap) * nth;
    double2* g = gbar + (size_t)((g0 + k) % gcap) * nth;
    double acc = 0.0;
    for (int j = 0; j < nth; ++j) {
        double2 v = w[j];
        acc += v.x * v.x + v.y * v.y;
        g[j] = make_double2(2.0 * r6 * v.x, 2.0 * r6 * v.y);
    }
    lossrec[k] = r6 * acc;
}

// out = sum of v[0 .. n) in index order (one thread: the order is part of the result).
__global__ void ordered_sum_kernel(const double* v, int64_t n, double* out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double acc = 0.0;
    for (int64_t k = 0; k < n; ++k) acc += v[k];
    *out = acc;
}

// ------------------------------------------------------------------ launchers

void launch_adj_init(cudaStream_t st, const InstDev& d, const double2* gbar, const CoLevel& out) {
    dim3 g(d.nr, (d.pitch + 127) / 128);
    if (d.prec == 0 || d.prec == 3) adj_init_kernel<double><<<g, 128, 0, st>>>(d, gbar, out);
    else adj_init_kernel<float><<<g, 128, 0, st>>>(d, gbar, out);
}

// dynamic shared memory of the reverse-step kernels for blocks of `threads` rows
template <typename R>
static size_t adj_smem(int threads, bool f32) {
    return 4 * (size_t)threads * sizeof(Z<R>) +
           (f32 ? 3 * (size_t)threads * sizeof(float4) + kAdjRtCols * sizeof(RTab2) : 0);
}

template <class K>
static int adj_resident(K kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

// f(kernel, dynamic shared memory) with the reverse-step kernel built for blocks of t rows
// (up to 256, 512 or 1024)
template <class F>
static void adj_dispatch(int prec, int t, F f) {
    if (prec == 0 || prec == 3) {
        const size_t sm = adj_smem<double>(t, false);
        if (prec == 0) {
            if (t <= 256) f(adj_step_kernel<double, double, 256>, sm);
            else if (t <= 512) f(adj_step_kernel<double, double, 512>, sm);
            else f(adj_step_kernel<double, double, 1024>, sm);
        } else {
            if (t <= 256) f(adj_step_kernel<DF, double, 256>, sm);
            else if (t <= 512) f(adj_step_kernel<DF, double, 512>, sm);
            else f(adj_step_kernel<DF, double, 1024>, sm);
        }
    } else {
        const size_t sm = adj_smem<float>(t, true);
        if (t <= 256) f(adj_step_kernel_f32<256>, sm);
        else if (t <= 512) f(adj_step_kernel_f32<512>, sm);
        else f(adj_step_kernel_f32<1024>, sm);
    }
}

int adj_step_plan(const InstDev& d, int* strip) {
    int res = 1;
    adj_dispatch(d.prec, d.pitch, [&](auto kernel, size_t sm) {
        // (blocks of more than 256 rows take more than the default 48 KB)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        res = adj_resident(kernel, d.pitch, sm);
    });
    int L = (d.nr + res - 1) / res;   // one wave of resident blocks, >= 4 columns each
    if (L < 4) L = 4;
    *strip = L;
    return (d.nr + L - 1) / L;
}

template <class K>
static void adj_launch(cudaStream_t st, K kernel, int nb, int t, size_t sm, const InstDev& d, const CoLevel& lin,
                       const double2* gbar, const CoLevel& lout, int strip, void* wh, void* wi) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(t);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, d, lin, gbar, lout, strip, wh, wi);
}

void launch_adj_step(cudaStream_t st, const InstDev& d, const CoLevel& lin, const double2* gbar,
                     const CoLevel& lout, int strip, void* wh, void* wi) {
    const int nb = (d.nr + strip - 1) / strip;
    adj_dispatch(d.prec, d.pitch, [&](auto kernel, size_t sm) {
        adj_launch(st, kernel, nb, d.pitch, sm, d, lin, gbar, lout, strip, wh, wi);
    });
}

size_t adj_window_bytes(const InstDev& d) {
    const size_t es = (d.prec == 0 || d.prec == 3) ? sizeof(double2) : sizeof(float2);
    return ((size_t)d.src.nh + d.src.ni) * d.src.nj * es;
}

void launch_adj_src_grad(cudaStream_t st, const InstDev& d, int64_t step0, int64_t k0, int64_t count,
                         int slots, const void* ring, double* gA, double* gR) {
    if (count <= 0) return;
    if (d.prec == 0 || d.prec == 3)
        adj_src_grad_kernel<double><<<(unsigned)count, kSrcGradThreads, 0, st>>>(d, step0, k0, slots, ring, gA, gR);
    else
        adj_src_grad_kernel<float><<<(unsigned)count, kSrcGradThreads, 0, st>>>(d, step0, k0, slots, ring, gA, gR);
}

void launch_loss_records(cudaStream_t st, const double2* wave, int64_t cap, int nth,
                         int64_t level0, int64_t count, double r6, double* lossrec,
                         double2* gbar, int64_t gcap, int64_t g0) {
    loss_records_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(wave, cap, nth, level0, count, r6,
                                                                        lossrec, gbar, gcap, g0);
}

void launch_ordered_sum(cudaStream_t st, const double* v, int64_t n, double* out) {
    ordered_sum_kernel<<<1, 32, 0, st>>>(v, n, out);
}

}  // namespace teuk
