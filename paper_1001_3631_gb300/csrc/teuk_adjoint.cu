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
// condition.  lam and mu are FP64 whatever the forward precision.
#include "teuk_internal.cuh"

namespace teuk {

struct Z { double x, y; };
__device__ __forceinline__ Z zld(const double2* p, size_t o) { double2 v = p[o]; return {v.x, v.y}; }
__device__ __forceinline__ Z zadd(Z a, Z b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ Z zscale(double s, Z a) { return {s * a.x, s * a.y}; }
// conj(cr + i ci) * z
__device__ __forceinline__ Z zconjmul(double cr, double ci, Z z) {
    return {cr * z.x + ci * z.y, cr * z.y - ci * z.x};
}

template <typename T>
__device__ __forceinline__ double cget(const T* tab, size_t pl, int k, size_t o) {
    return (double)tab[(size_t)k * pl + o];
}

// Cotangent of the averaged Phi~ at (col, j) produced by the angular term of the
// sub-step whose coefficients are `tab` and whose Pi cotangents are L (col fixed).
template <typename T>
__device__ __forceinline__ Z theta_cotangent(const T* tab, size_t pl, const double2* LP,
                                             const InstDev& d, int col, int j, double g) {
    const int nth = d.nth;
    size_t o = node_index(d, col, j);
    Z l0 = zld(LP, o);
    double ep0 = cget(tab, pl, C_EP, o), em0 = cget(tab, pl, C_EM, o);
    Z r = zconjmul(cget(tab, pl, C_E3R, o) - ep0 - em0, cget(tab, pl, C_E3I, o), l0);
    if (j >= 1) {
        size_t om = o - 1;   // row j-1
        r = zadd(r, zscale(cget(tab, pl, C_EP, om), zld(LP, om)));
    } else {
        r = zadd(r, zscale(g * em0, l0));   // ghost row -1 = g * row 0
    }
    if (j + 1 < nth) {
        size_t op = o + 1;   // row j+1
        r = zadd(r, zscale(cget(tab, pl, C_EM, op), zld(LP, op)));
    } else {
        r = zadd(r, zscale(g * ep0, l0));   // ghost row nth = g * row nth-1
    }
    return r;
}

// mu = C^T P lam  at half node (h, j), h in [0, nr-2].
template <typename T>
__global__ void adj_corrector_kernel(InstDev d, const double2* lF, const double2* lP, double2* mF,
                                     double2* mP) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int h = blockIdx.y;
    if (h > d.nr - 2 || j >= d.nth) return;
    const T* ci = (const T*)d.coef_i;
    const size_t pl = plane_elems(d);
    Z muF = {0, 0}, muP = {0, 0};
    // integer node h (this half node is its right neighbour R, sign +1) and
    // integer node h+1 (this half node is its left neighbour L, sign -1)
    for (int side = 0; side < 2; ++side) {
        int col = h + side;
        if (col < 1 || col > d.nr - 2) continue;   // P: boundary columns carry no cotangent
        double sR = side == 0 ? 1.0 : -1.0;
        size_t o = node_index(d, col, j);
        Z LF = zld(lF, o), LPi = zld(lP, o);
        double G = cget(ci, pl, C_G, o);
        Z tc = theta_cotangent<T>(ci, pl, lP, d, col, j, d.ghost);
        // Delta Phi = -G (hF_R - hF_L) + dt (hP_R + hP_L)/2
        // Delta Pi  =  G (hP_R - hP_L) + E1 (hP_R + hP_L)/2 + E2 (hF_R - hF_L) + angular(Phi~)
        muF = zadd(muF, zscale(-sR * G, LF));
        muF = zadd(muF, zscale(sR, zconjmul(cget(ci, pl, C_E2R, o), cget(ci, pl, C_E2I, o), LPi)));
        muF = zadd(muF, zscale(0.5, tc));
        muP = zadd(muP, zscale(0.5 * d.dt, LF));
        muP = zadd(muP, zscale(sR * G, LPi));
        muP = zadd(muP, zscale(0.5, zconjmul(cget(ci, pl, C_E1R, o), cget(ci, pl, C_E1I, o), LPi)));
    }
    size_t oh = node_index(d, h, j);
    mF[oh] = make_double2(muF.x, muF.y);
    mP[oh] = make_double2(muP.x, muP.y);
}

// lam^n = P lam^{n+1} + H^T mu (+ E^T gbar) at node (i, j).
template <typename T>
__global__ void adj_predictor_kernel(InstDev d, const double2* lF, const double2* lP,
                                     const double2* mF, const double2* mP, const double2* gbar,
                                     double2* oF, double2* oP) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (i >= d.nr || j >= d.nth) return;
    const T* ch = (const T*)d.coef_h;
    const size_t pl = plane_elems(d);
    const size_t o = node_index(d, i, j);
    const bool interior = i >= 1 && i <= d.nr - 2;
    Z aF = interior ? zld(lF, o) : Z{0, 0};
    Z aP = interior ? zld(lP, o) : Z{0, 0};
    const double hdt = 0.5 * d.dt;
    // half node i-1/2 (index i-1, this column is its right input R, sign +1) and
    // half node i+1/2 (index i, this column is its left input L, sign -1)
    for (int side = 0; side < 2; ++side) {
        int h = i - 1 + side;
        if (h < 0 || h > d.nr - 2) continue;
        double sR = side == 0 ? 1.0 : -1.0;
        size_t oh = node_index(d, h, j);
        Z MF = zld(mF, oh), MP = zld(mP, oh);
        double G = cget(ch, pl, C_G, oh);
        Z tc = theta_cotangent<T>(ch, pl, mP, d, h, j, d.ghost);
        // hF = (F_L + F_R)/2 - G (F_R - F_L) + hdt (P_L + P_R)/2
        // hP = (P_L + P_R)/2 + G (P_R - P_L) + E1 (P_L + P_R)/2 + E2 (F_R - F_L) + angular(Fbar)
        aF = zadd(aF, zscale(0.5 - sR * G, MF));
        aF = zadd(aF, zscale(sR, zconjmul(cget(ch, pl, C_E2R, oh), cget(ch, pl, C_E2I, oh), MP)));
        aF = zadd(aF, zscale(0.5, tc));
        aP = zadd(aP, zscale(0.5 * hdt, MF));
        aP = zadd(aP, zscale(0.5 + sR * G, MP));
        aP = zadd(aP, zscale(0.5, zconjmul(cget(ch, pl, C_E1R, oh), cget(ch, pl, C_E1I, oh), MP)));
    }
    if (gbar) {  // transpose of the linear extraction between i_e and i_e + 1
        if (i == d.i_e) aF = zadd(aF, zscale(1.0 - d.f_e, zld(gbar, j)));
        if (i == d.i_e + 1) aF = zadd(aF, zscale(d.f_e, zld(gbar, j)));
    }
    oF[o] = make_double2(aF.x, aF.y);
    oP[o] = make_double2(aP.x, aP.y);
}

// lam = E^T gbar (the start of the reverse sweep).
__global__ void adj_init_kernel(InstDev d, const double2* gbar, double2* oF, double2* oP) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= d.pitch || i >= d.nr) return;
    size_t o = node_index(d, i, j);
    Z a = {0, 0};
    if (gbar && i == d.i_e) a = zscale(1.0 - d.f_e, zld(gbar, j));
    if (gbar && i == d.i_e + 1) a = zscale(d.f_e, zld(gbar, j));
    oF[o] = make_double2(a.x, a.y);
    oP[o] = make_double2(0.0, 0.0);
}

// Source gradients of step n: one block, fixed-order reduction.
__global__ void adj_source_kernel(InstDev d, int64_t n, const double2* lP, const double2* mP,
                                  double* gA, double* gR) {
    __shared__ double sA[256], sR[256];
    const SourceDev& s = d.src;
    double A = (s.amps != nullptr && n < s.n_amps) ? s.amps[n] : 1.0;
    double tp = (double)n * d.dt, tc = tp + 0.5 * d.dt;
    double sp, cp, sc, cc;
    sincos(s.omega * tp + s.phase0, &sp, &cp);
    sincos(s.omega * tc + s.phase0, &sc, &cc);
    Z ep = {cp, -sp}, ec = {cc, -sc};
    // d/dr0 e^{-i phi} = -i (dphi/dr0) e^{-i phi}
    double kp = tp * s.domega + s.dphase0, kc = tc * s.domega + s.dphase0;
    // (-i k)(x + i y) = k y - i k x
    Z dep = {kp * ep.y, -kp * ep.x}, dec = {kc * ec.y, -kc * ec.x};
    double accA = 0.0, accR = 0.0;
    const double hdt = 0.5 * d.dt;
    int nh_tot = s.nj * s.nh, ni_tot = s.nj * s.ni;
    for (int k = threadIdx.x; k < nh_tot + ni_tot; k += blockDim.x) {
        Z lam, P, dP, e, de;
        double w;
        if (k < nh_tot) {
            int jj = k / s.nh, hh = k % s.nh;
            size_t o = node_index(d, s.h_lo + hh, s.j_lo + jj);
            lam = zld(mP, o);
            P = {s.P_half[k].x, s.P_half[k].y};
            dP = {s.dP_half[k].x, s.dP_half[k].y};
            e = ep; de = dep; w = hdt;
        } else {
            int kk = k - nh_tot;
            int jj = kk / s.ni, ii = kk % s.ni;
            int col = s.i_lo + ii;
            if (col < 1 || col > d.nr - 2) continue;
            size_t o = node_index(d, col, s.j_lo + jj);
            lam = zld(lP, o);
            P = {s.P_int[kk].x, s.P_int[kk].y};
            dP = {s.dP_int[kk].x, s.dP_int[kk].y};
            e = ec; de = dec; w = d.dt;
        }
        // e P and (de P + e dP)
        Z eP = {e.x * P.x - e.y * P.y, e.x * P.y + e.y * P.x};
        Z dd = {de.x * P.x - de.y * P.y + e.x * dP.x - e.y * dP.y,
                de.x * P.y + de.y * P.x + e.x * dP.y + e.y * dP.x};
        accA += w * (lam.x * eP.x + lam.y * eP.y);
        accR += w * (lam.x * dd.x + lam.y * dd.y);
    }
    sA[threadIdx.x] = accA;
    sR[threadIdx.x] = accR;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sA[threadIdx.x] += sA[threadIdx.x + st];
            sR[threadIdx.x] += sR[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *gA = sA[0];
        *gR = A * sR[0];
    }
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

void launch_adj_corrector(cudaStream_t st, const InstDev& d, const double2* lF, const double2* lP,
                          double2* mF, double2* mP) {
    dim3 g((d.nth + 127) / 128, d.nr - 1);
    if (d.prec == 0) adj_corrector_kernel<double><<<g, 128, 0, st>>>(d, lF, lP, mF, mP);
    else adj_corrector_kernel<float><<<g, 128, 0, st>>>(d, lF, lP, mF, mP);
}

void launch_adj_predictor(cudaStream_t st, const InstDev& d, const double2* lF, const double2* lP,
                          const double2* mF, const double2* mP, const double2* gbar, double2* oF,
                          double2* oP) {
    dim3 g((d.nth + 127) / 128, d.nr);
    if (d.prec == 0)
        adj_predictor_kernel<double><<<g, 128, 0, st>>>(d, lF, lP, mF, mP, gbar, oF, oP);
    else
        adj_predictor_kernel<float><<<g, 128, 0, st>>>(d, lF, lP, mF, mP, gbar, oF, oP);
}

void launch_adj_init(cudaStream_t st, const InstDev& d, const double2* gbar, double2* oF,
                     double2* oP) {
    dim3 g((d.pitch + 127) / 128, d.nr);
    adj_init_kernel<<<g, 128, 0, st>>>(d, gbar, oF, oP);
}

void launch_adj_source(cudaStream_t st, const InstDev& d, int64_t n, const double2* lP,
                       const double2* mP, double* gA, double* gR) {
    adj_source_kernel<<<1, 256, 0, st>>>(d, n, lP, mP, gA, gR);
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
