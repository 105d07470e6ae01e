// teuk_adjoint.cu -- transpose of one Lax-Wendroff step (Eqs. 13-14), as gathers.
//
// The step is affine and complex-linear in u:  u^{n+1} = P (u^n + C(H u^n)) + A_n s_n,
// with H the predictor of Eq. (13) (integer nodes -> half nodes), C the corrector
// increment of Eq. (14) (half nodes -> integer nodes) and P the radial boundary
// condition (zero at i = 0 and i = n_rstar - 1).  With the real inner product
// <x, y> = sum Re(conj(x) y), the transpose of y += c x is x += conj(c) y.  So one
// reverse step is
//   lam'  = P lam^{n+1}
//   mu    = C^T lam'                       (adj_corrector_kernel, one thread per half node)
//   lam^n = lam' + H^T mu + E^T gbar_n     (adj_predictor_kernel, one thread per node)
// and the source enters the gradients as
//   dL/dA_n  = <mu_Pi, (dt/2) e_p P_half> + <lam'_Pi, dt e_c P_int>
//   dL/dr0  += A_n (<mu_Pi, (dt/2) d(e_p P_half)/dr0> + <lam'_Pi, dt d(e_c P_int)/dr0>)
// with e_p = e^{-i(omega t_n + phase0)}, e_c the same at t_n + dt/2
// (adj_source_kernel, one block per step, fixed reduction order).
// Coefficients are the scaled tables of teuk_setup.cu (g, E1, E2, ep, em, E3); in
// the corrector's angular term  ep Phi~(j+1) + em Phi~(j-1) + (E3 - ep - em) Phi~(j)
// the ghost rows fold back onto rows 0 and n_theta-1 with the sign of the pole
// condition.  The co-state lam and mu are FP64 for FP64 instances; for FP32 instances
// they are FP32, lam compensated like the forward state (value hi - c, each step's
// increment added with Kahan's compensated sum), the gradient sums FP64 either way.
#include <type_traits>

#include "teuk_df.cuh"
#include "teuk_internal.cuh"

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

// Cotangent of the averaged Phi~ at (col, j) produced by the angular term of the
// sub-step whose coefficients are `tab` and whose Pi cotangents are LP (col fixed).
template <typename T, typename R, class LD>
__device__ __forceinline__ Z<R> theta_cotangent(const T* tab, size_t pl, const LD& LP,
                                                const InstDev& d, int col, int j, R g) {
    const int nth = d.nth;
    size_t o = node_index(d, col, j);
    Z<R> l0 = LP(o);
    R ep0 = cget<T, R>(tab, pl, C_EP, o), em0 = cget<T, R>(tab, pl, C_EM, o);
    Z<R> r = zconjmul(cget<T, R>(tab, pl, C_E3R, o) - ep0 - em0, cget<T, R>(tab, pl, C_E3I, o), l0);
    if (j >= 1) {
        size_t om = o - 1;   // row j-1
        r = zadd(r, zscale(cget<T, R>(tab, pl, C_EP, om), LP(om)));
    } else {
        r = zadd(r, zscale(g * em0, l0));   // ghost row -1 = g * row 0
    }
    if (j + 1 < nth) {
        size_t op = o + 1;   // row j+1
        r = zadd(r, zscale(cget<T, R>(tab, pl, C_EM, op), LP(op)));
    } else {
        r = zadd(r, zscale(g * ep0, l0));   // ghost row nth = g * row nth-1
    }
    return r;
}

// mu = C^T P lam  at half node (h, j), h in [0, nr-2].
template <typename T, typename R>
__global__ void adj_corrector_kernel(InstDev d, CoLevel lam, CoMu mu) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int h = blockIdx.y;
    if (h > d.nr - 2 || j >= d.nth) return;
    const T* ci = (const T*)d.coef_i;
    const size_t pl = plane_elems(d);
    const CoPlane<R> lF = coplane<R>(lam, 0), lP = coplane<R>(lam, 1);
    auto LPf = [&](size_t o) { return lP.ld(o); };
    Z<R> muF = {0, 0}, muP = {0, 0};
    // integer node h (this half node is its right neighbour R, sign +1) and
    // integer node h+1 (this half node is its left neighbour L, sign -1)
    for (int side = 0; side < 2; ++side) {
        int col = h + side;
        if (col < 1 || col > d.nr - 2) continue;   // P: boundary columns carry no cotangent
        R sR = side == 0 ? R(1) : R(-1);
        size_t o = node_index(d, col, j);
        Z<R> LF = lF.ld(o), LPi = lP.ld(o);
        R G = cget<T, R>(ci, pl, C_G, o);
        Z<R> tc = theta_cotangent<T, R>(ci, pl, LPf, d, col, j, (R)d.ghost);
        // Delta Phi = -G (hF_R - hF_L) + dt (hP_R + hP_L)/2
        // Delta Pi  =  G (hP_R - hP_L) + E1 (hP_R + hP_L)/2 + E2 (hF_R - hF_L) + angular(Phi~)
        muF = zadd(muF, zscale(-sR * G, LF));
        muF = zadd(muF, zscale(sR, zconjmul(cget<T, R>(ci, pl, C_E2R, o), cget<T, R>(ci, pl, C_E2I, o), LPi)));
        muF = zadd(muF, zscale(R(0.5), tc));
        muP = zadd(muP, zscale((R)(0.5 * d.dt), LF));
        muP = zadd(muP, zscale(sR * G, LPi));
        muP = zadd(muP, zscale(R(0.5), zconjmul(cget<T, R>(ci, pl, C_E1R, o), cget<T, R>(ci, pl, C_E1I, o), LPi)));
    }
    size_t oh = node_index(d, h, j);
    stv<R>(mu.F, oh, muF);
    stv<R>(mu.P, oh, muP);
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

// lam^n = P lam^{n+1} + H^T mu (+ E^T gbar) at node (i, j).
template <typename T, typename R>
__global__ void adj_predictor_kernel(InstDev d, CoLevel lin, CoMu mu, const double2* gbar,
                                     CoLevel lout) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (i >= d.nr || j >= d.nth) return;
    const T* ch = (const T*)d.coef_h;
    const size_t pl = plane_elems(d);
    const size_t o = node_index(d, i, j);
    const bool interior = i >= 1 && i <= d.nr - 2;
    constexpr bool kComp = sizeof(R) == 4;
    // FP64: the sum starts from P lam^{n+1}; FP32: the increment alone, added to the
    // compensated lam^{n+1} at the end
    Z<R> aF = {0, 0}, aP = {0, 0};
    if constexpr (!kComp) {
        if (interior) {
            aF = ldv<R>(lin.F, o);
            aP = ldv<R>(lin.P, o);
        }
    }
    const R hdt = (R)(0.5 * d.dt);
    auto MPf = [&](size_t q) { return ldv<R>(mu.P, q); };
    // half node i-1/2 (index i-1, this column is its right input R, sign +1) and
    // half node i+1/2 (index i, this column is its left input L, sign -1)
    for (int side = 0; side < 2; ++side) {
        int h = i - 1 + side;
        if (h < 0 || h > d.nr - 2) continue;
        R sR = side == 0 ? R(1) : R(-1);
        size_t oh = node_index(d, h, j);
        Z<R> MF = ldv<R>(mu.F, oh), MP = ldv<R>(mu.P, oh);
        R G = cget<T, R>(ch, pl, C_G, oh);
        Z<R> tc = theta_cotangent<T, R>(ch, pl, MPf, d, h, j, (R)d.ghost);
        // hF = (F_L + F_R)/2 - G (F_R - F_L) + hdt (P_L + P_R)/2
        // hP = (P_L + P_R)/2 + G (P_R - P_L) + E1 (P_L + P_R)/2 + E2 (F_R - F_L) + angular(Fbar)
        aF = zadd(aF, zscale(R(0.5) - sR * G, MF));
        aF = zadd(aF, zscale(sR, zconjmul(cget<T, R>(ch, pl, C_E2R, oh), cget<T, R>(ch, pl, C_E2I, oh), MP)));
        aF = zadd(aF, zscale(R(0.5), tc));
        aP = zadd(aP, zscale(R(0.5) * hdt, MF));
        aP = zadd(aP, zscale(R(0.5) + sR * G, MP));
        aP = zadd(aP, zscale(R(0.5), zconjmul(cget<T, R>(ch, pl, C_E1R, oh), cget<T, R>(ch, pl, C_E1I, oh), MP)));
    }
    if (gbar) {  // transpose of the linear extraction between i_e and i_e + 1
        if (i == d.i_e) aF = zadd(aF, zscale((R)(1.0 - d.f_e), gld<R>(gbar, j)));
        if (i == d.i_e + 1) aF = zadd(aF, zscale((R)d.f_e, gld<R>(gbar, j)));
    }
    if constexpr (kComp) {
        float2 vF = {0.f, 0.f}, cF = {0.f, 0.f}, vP = {0.f, 0.f}, cP = {0.f, 0.f};
        if (interior) {
            vF = ((const float2*)lin.F)[o];
            cF = ((const float2*)lin.Fc)[o];
            vP = ((const float2*)lin.P)[o];
            cP = ((const float2*)lin.Pc)[o];
        }
        kahan_node(vF, cF, aF);
        kahan_node(vP, cP, aP);
        ((float2*)lout.F)[o] = vF;
        ((float2*)lout.Fc)[o] = cF;
        ((float2*)lout.P)[o] = vP;
        ((float2*)lout.Pc)[o] = cP;
    } else {
        stv<R>(lout.F, o, aF);
        stv<R>(lout.P, o, aP);
    }
}

// lam = E^T gbar (the start of the reverse sweep).
template <typename R>
__global__ void adj_init_kernel(InstDev d, const double2* gbar, CoLevel out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
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

// Source gradients of step n.  With e = e^{-i phi} the phase of a sub-step and
// de = d e / d r0,
//   dL/dA_n  = Re( (dt/2) e_p S_h + dt e_c S_i ),
//   dL/dr0  += A_n Re( (dt/2) (de_p S_h + e_p S'_h) + dt (de_c S_i + e_c S'_i) ),
// where S_h = sum conj(mu_Pi) P_half and S'_h = sum conj(mu_Pi) dP_half over the
// half-node window, S_i and S'_i the same with lam'_Pi over the integer-node window
// (interior columns only).  The four complex sums are FP64: each block reduces a fixed
// slice of the window in a fixed order, and the last block to finish adds the blocks'
// partial sums in index order and applies the phases, so the result does not depend
// on the scheduling.
constexpr int kSrcThreads = 256;
template <typename R>
__global__ void adj_source_kernel(InstDev d, int64_t n, CoLevel lam, CoMu mu, double* part,
                                  unsigned* done, double* gA, double* gR) {
    __shared__ double red[8][kSrcThreads];
    __shared__ bool last;
    const SourceDev& s = d.src;
    const CoPlane<R> lP = coplane<R>(lam, 1);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // S_h, S'_h, S_i, S'_i (re, im)
    const int nh_tot = s.nj * s.nh, ni_tot = s.nj * s.ni;
    const int stride = gridDim.x * kSrcThreads;
    for (int k = blockIdx.x * kSrcThreads + threadIdx.x; k < nh_tot + ni_tot; k += stride) {
        Z<double> l, P, dP;
        int q;
        if (k < nh_tot) {
            int jj = k / s.nh, hh = k % s.nh;
            const Z<R> m = ldv<R>(mu.P, node_index(d, s.h_lo + hh, s.j_lo + jj));
            l = {(double)m.x, (double)m.y};
            P = {s.P_half[k].x, s.P_half[k].y};
            dP = {s.dP_half[k].x, s.dP_half[k].y};
            q = 0;
        } else {
            int kk = k - nh_tot;
            int jj = kk / s.ni, ii = kk % s.ni;
            int col = s.i_lo + ii;
            if (col < 1 || col > d.nr - 2) continue;
            const Z<R> v = lP.ld(node_index(d, col, s.j_lo + jj));
            l = {(double)v.x, (double)v.y};
            P = {s.P_int[kk].x, s.P_int[kk].y};
            dP = {s.dP_int[kk].x, s.dP_int[kk].y};
            q = 4;
        }
        // conj(l) P and conj(l) dP
        acc[q + 0] += l.x * P.x + l.y * P.y;
        acc[q + 1] += l.x * P.y - l.y * P.x;
        acc[q + 2] += l.x * dP.x + l.y * dP.y;
        acc[q + 3] += l.x * dP.y - l.y * dP.x;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int st = kSrcThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int v = 0; v < 8; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int v = 0; v < 8; ++v) part[blockIdx.x * 8 + v] = red[v][0];
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: threads 0..7 each add one of the eight sums over the blocks in
    // index order; threads 32 and 64 form the two phases meanwhile
    __shared__ double S[8];
    __shared__ Z<double> ph[4];   // e_p, e_c, de_p, de_c
    const int t = threadIdx.x;
    if (t < 8) {
        double acc_v = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) acc_v += ((volatile double*)part)[b * 8 + t];
        S[t] = acc_v;
    }
    if (t == 32 || t == 64) {
        const double tt = (double)n * d.dt + (t == 32 ? 0.0 : 0.5 * d.dt);
        double sn, cs;
        sincos(s.omega * tt + s.phase0, &sn, &cs);
        // e = (cos, -sin); de = -i k e with k = d phi / d r0
        const double k = tt * s.domega + s.dphase0;
        const Z<double> e = {cs, -sn};
        ph[t == 32 ? 0 : 1] = e;
        ph[t == 32 ? 2 : 3] = Z<double>{k * e.y, -k * e.x};
    }
    __syncthreads();
    if (t != 0) return;
    *done = 0;   // ready for the next step's launch (stream-ordered)
    const double A = (s.amps != nullptr && n < s.n_amps) ? s.amps[n] : 1.0;
    auto re_mul = [](Z<double> a, double bx, double by) { return a.x * bx - a.y * by; };
    const double hdt = 0.5 * d.dt;
    *gA = hdt * re_mul(ph[0], S[0], S[1]) + d.dt * re_mul(ph[1], S[4], S[5]);
    *gR = A * (hdt * (re_mul(ph[2], S[0], S[1]) + re_mul(ph[0], S[2], S[3])) +
               d.dt * (re_mul(ph[3], S[4], S[5]) + re_mul(ph[1], S[6], S[7])));
}

// Loss of the built-in |r_ext^3 W|^2: per record, lossrec[k] = r^6 sum_j |W_k[j]|^2 (j
// ascending) and gbar_k = 2 r^6 W_k.  Records are read from a ring (slot level % cap).
__global__ void loss_records_kernel(const double2* wave, int64_t cap, int nth, int64_t level0,
                                    int64_t count, double r6, double* lossrec, double2* gbar) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    const double2* w = wave + (size_t)((level0 + k) % cap) * nth;
    double acc = 0.0;
    for (int j = 0; j < nth; ++j) {
        double2 v = w[j];
        acc += v.x * v.x + v.y * v.y;
        gbar[(size_t)k * nth + j] = make_double2(2.0 * r6 * v.x, 2.0 * r6 * v.y);
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

void launch_adj_corrector(cudaStream_t st, const InstDev& d, const CoLevel& lam, const CoMu& mu) {
    dim3 g((d.nth + 127) / 128, d.nr - 1);
    if (d.prec == 0) adj_corrector_kernel<double, double><<<g, 128, 0, st>>>(d, lam, mu);
    else if (d.prec == 3) adj_corrector_kernel<DF, double><<<g, 128, 0, st>>>(d, lam, mu);
    else adj_corrector_kernel<float, float><<<g, 128, 0, st>>>(d, lam, mu);
}

void launch_adj_predictor(cudaStream_t st, const InstDev& d, const CoLevel& lin, const CoMu& mu,
                          const double2* gbar, const CoLevel& lout) {
    dim3 g((d.nth + 127) / 128, d.nr);
    if (d.prec == 0) adj_predictor_kernel<double, double><<<g, 128, 0, st>>>(d, lin, mu, gbar, lout);
    else if (d.prec == 3) adj_predictor_kernel<DF, double><<<g, 128, 0, st>>>(d, lin, mu, gbar, lout);
    else adj_predictor_kernel<float, float><<<g, 128, 0, st>>>(d, lin, mu, gbar, lout);
}

void launch_adj_init(cudaStream_t st, const InstDev& d, const double2* gbar, const CoLevel& out) {
    dim3 g((d.pitch + 127) / 128, d.nr);
    if (d.prec == 0 || d.prec == 3) adj_init_kernel<double><<<g, 128, 0, st>>>(d, gbar, out);
    else adj_init_kernel<float><<<g, 128, 0, st>>>(d, gbar, out);
}

int adj_source_blocks(const InstDev& d) {
    const int tot = d.src.nj * (d.src.nh + d.src.ni);
    const int b = (tot + kSrcThreads - 1) / kSrcThreads;
    return b < 1 ? 1 : (b > kAdjSourceMaxBlocks ? kAdjSourceMaxBlocks : b);
}

void launch_adj_source(cudaStream_t st, const InstDev& d, int64_t n, const CoLevel& lam,
                       const CoMu& mu, double* part, unsigned* done, double* gA, double* gR) {
    const int nb = adj_source_blocks(d);
    if (d.prec == 0 || d.prec == 3)
        adj_source_kernel<double><<<nb, kSrcThreads, 0, st>>>(d, n, lam, mu, part, done, gA, gR);
    else adj_source_kernel<float><<<nb, kSrcThreads, 0, st>>>(d, n, lam, mu, part, done, gA, gR);
}

void launch_loss_records(cudaStream_t st, const double2* wave, int64_t cap, int nth,
                         int64_t level0, int64_t count, double r6, double* lossrec,
                         double2* gbar) {
    loss_records_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(wave, cap, nth, level0,
                                                                        count, r6, lossrec, gbar);
}

void launch_ordered_sum(cudaStream_t st, const double* v, int64_t n, double* out) {
    ordered_sum_kernel<<<1, 32, 0, st>>>(v, n, out);
}

}  // namespace teuk
