// teuk_setup.cu -- one-time setup kernels (FP64): tortoise inversion, coefficient
// tables and the source profile.
//
// Coefficients of the first-order system d_t u + D d_r* u = S (Eqs. 8-12), obtained
// from Eq. (1) by the substitutions of Eqs. (2)-(7):
//   S_Phi = Pi
//   S_Pi  = -c_t Pi + P* Phi_* + w Theta[Phi] + q Phi + tau
// with R = r^2 + a^2, Sigma^2 = R^2 - a^2 Delta sin^2 (Eq. 7), b = R/Sigma (Eq. 6),
//   w   = Delta / Sigma^2
//   c_t = [4 i M a m r + 2 s (r Delta - M (r^2 - a^2)) + 2 i s a Delta cos] / Sigma^2
//   p*  = w (6 R / r + 2 r) + 2 R (s (r - M) + i m a) / Sigma^2
//   q   = [6 Delta^2/r^2 + 6 Delta ((s+1)(r-M) + i m a)/r + 4 i s m a (r - M)] / Sigma^2
//   b b_{,r*} = a^2 Delta sin^2 (2 R (r - M) - 4 r Delta) / (2 Sigma^4)
//   P*  = c_t b + p* - b b_{,r*}
//   Theta[F] = F_thth + cot F_th - V F,  V = (m + s cos)^2 / sin^2 - s
// evaluated at r = r_+ + x with x from the inversion of Eq. (2), so that
// Delta = x (x + r_+ - r_-) keeps full relative precision next to the horizon.
#include "teuk_df.cuh"
#include "teuk_internal.cuh"

namespace teuk {

__device__ __forceinline__ double rstar_of_x(double M, double rp, double rm, double x) {
    double k = 2.0 * M / (rp - rm);
    double r = rp + x;
    return r + k * rp * log(x / (2.0 * M)) - k * rm * log((r - rm) / (2.0 * M));
}

// Solve r*(r_+ + x) = target for x > 0: safeguarded Newton in y = ln x.
// dr*/dy = x dr*/dr = x R / Delta = R / (x + r_+ - r_-).
__device__ double x_of_rstar(double M, double a, double target) {
    double d = sqrt(M * M - a * a);
    double rp = M + d, rm = M - d;
    double lo = -700.0, hi = 30.0;
    double k = 2.0 * M * rp / (rp - rm);
    // initial guess from the two asymptotes (far: r* ~ r, near horizon: r* ~ k ln x)
    double y = target > rp + 4.0 ? log(target) : (target - rp) / k;
    y = fmin(fmax(y, lo + 1.0), hi - 1.0);
    for (int it = 0; it < 200; ++it) {
        double x = exp(y);
        double f = rstar_of_x(M, rp, rm, x) - target;
        if (f > 0.0) hi = y; else lo = y;
        double r = rp + x;
        double fp = (r * r + a * a) / (x + rp - rm);
        double yn = y - f / fp;
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);  // keep the bracket
        if (fabs(yn - y) <= 1e-15 * fmax(1.0, fabs(y))) { y = yn; break; }
        y = yn;
    }
    return exp(y);
}

// Node k of the instance is node k + off of its grid (off > 0 for a slab of a larger grid).
__global__ void invert_tortoise_kernel(double M, double a, double rstar_min, double drs, int nr,
                                       int off, double* x_int, double* x_half) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nr) x_int[k] = x_of_rstar(M, a, rstar_min + (k + off) * drs);
    if (k < nr - 1) x_half[k] = x_of_rstar(M, a, rstar_min + ((k + off) + 0.5) * drs);
}

struct Cplx { double re, im; };

// The nine scaled coefficients (order of CoefIdx) of a sub-step that spans the
// fraction sfrac of dt, at (r = r_+ + x, theta).
__device__ void node_coefficients(double M, double a, int s_, int m_, double x, double th,
                                  double dth, double dt, double drs, double sfrac, double* out) {
    double d = sqrt(M * M - a * a);
    double rp = M + d, rm = M - d;
    double s = (double)s_, m = (double)m_;
    double r = rp + x;
    double Delta = x * (x + rp - rm);
    double R = r * r + a * a;
    double sn, cs;
    sincos(th, &sn, &cs);
    double sn2 = sn * sn;
    double Sig2 = R * R - a * a * Delta * sn2;
    double iS2 = 1.0 / Sig2;
    double b = R / sqrt(Sig2);
    double w = Delta * iS2;
    Cplx ct = {2.0 * s * (r * Delta - M * (r * r - a * a)) * iS2,
               (4.0 * M * a * m * r + 2.0 * s * a * Delta * cs) * iS2};
    Cplx pst = {w * (6.0 * R / r + 2.0 * r) + 2.0 * R * s * (r - M) * iS2,
                2.0 * R * m * a * iS2};
    Cplx q = {(6.0 * Delta * Delta / (r * r) + 6.0 * Delta * (s + 1.0) * (r - M) / r) * iS2,
              (6.0 * Delta * m * a / r + 4.0 * s * m * a * (r - M)) * iS2};
    double bbr = a * a * Delta * sn2 * (2.0 * R * (r - M) - 4.0 * r * Delta) * 0.5 * iS2 * iS2;
    Cplx Pst = {ct.re * b + pst.re - bbr, ct.im * b + pst.im};
    double V = (m + s * cs) * (m + s * cs) / sn2 - s;
    double cot = cs / sn;
    double sdt = sfrac * dt;
    double i2 = 1.0 / (dth * dth), i1 = cot / (2.0 * dth);
    out[C_G] = sdt * b / drs;
    out[C_E1R] = -sdt * ct.re;
    out[C_E1I] = -sdt * ct.im;
    out[C_E2R] = sdt * Pst.re / drs;
    out[C_E2I] = sdt * Pst.im / drs;
    out[C_EP] = sdt * w * (i2 + i1);
    out[C_EM] = sdt * w * (i2 - i1);
    out[C_E3R] = sdt * (q.re - w * V);
    out[C_E3I] = sdt * q.im;
}

template <typename T>
__global__ void coef_kernel(double M, double a, int s, int m, double rstar_min, double drs,
                            double dth, double dt, int nr, int nth, int pitch,
                            const double* x_int, const double* x_half, T* coef_h, T* coef_i) {
    int j = blockIdx.y * blockDim.x + threadIdx.x;   // theta row (fastest in memory)
    int i = blockIdx.x;                              // r* column (grid x: up to 2^31 - 1)
    if (j >= pitch || i >= nr) return;
    size_t pl = (size_t)nr * pitch;
    size_t o = (size_t)i * pitch + j;
    double th = (j + 0.5) * dth;
    double c[kNCoef];
    if (j < nth && i < nr - 1) {
        node_coefficients(M, a, s, m, x_half[i], th, dth, dt, drs, 0.5, c);
        for (int k = 0; k < kNCoef; ++k) coef_h[k * pl + o] = (T)c[k];
    } else {
        for (int k = 0; k < kNCoef; ++k) coef_h[k * pl + o] = (T)0;
    }
    if (j < nth) {
        node_coefficients(M, a, s, m, x_int[i], th, dth, dt, drs, 1.0, c);
        for (int k = 0; k < kNCoef; ++k) coef_i[k * pl + o] = (T)c[k];
    } else {
        for (int k = 0; k < kNCoef; ++k) coef_i[k * pl + o] = (T)0;
    }
}

// Source profile on the window: P = 4 pi (r^2 + a^2 cos^2) Delta / (Sigma^2 r^3) * G,
// G = exp(-(dr^2/sig_r^2 + dth^2/sig_t^2)/2) / (2 pi sig_r sig_t), zero beyond 8 sigma;
// dP/dr0 = P (r* - r*0)/sig_r^2 * dr*0/dr0 (widths fixed in cells or absolute units).
__device__ void profile_point(double M, double a, double x, double rs, double th, double rs0,
                              double sig_r, double sig_t, double drs0_dr0, double2* P,
                              double2* dP) {
    double dr = rs - rs0, dtt = th - 0.5 * 3.141592653589793238462643;
    if (fabs(dr) > 8.0 * sig_r || fabs(dtt) > 8.0 * sig_t) {
        *P = make_double2(0.0, 0.0);
        *dP = make_double2(0.0, 0.0);
        return;
    }
    double d = sqrt(M * M - a * a);
    double rp = M + d, rm = M - d;
    double r = rp + x;
    double Delta = x * (x + rp - rm);
    double R = r * r + a * a;
    double sn, cs;
    sincos(th, &sn, &cs);
    double Sig2 = R * R - a * a * Delta * sn * sn;
    double G = exp(-0.5 * (dr * dr / (sig_r * sig_r) + dtt * dtt / (sig_t * sig_t))) /
               (2.0 * 3.141592653589793238462643 * sig_r * sig_t);
    double pref = 4.0 * 3.141592653589793238462643 * (r * r + a * a * cs * cs) * Delta /
                  (Sig2 * r * r * r);
    *P = make_double2(pref * G, 0.0);
    *dP = make_double2(pref * G * dr / (sig_r * sig_r) * drs0_dr0, 0.0);
}

// One complex value into a profile in the arithmetic type of precision prec (double2;
// double-float re.hi, re.lo, im.hi, im.lo; float2)
__device__ __forceinline__ void put_cplx(const void* q, size_t idx, double2 v, int prec) {
    if (prec == 0) {
        ((double2*)q)[idx] = v;
    } else if (prec == 3) {
        const DF x(v.x), y(v.y);
        ((float4*)q)[idx] = make_float4(x.hi, x.lo, y.hi, y.lo);
    } else {
        ((float2*)q)[idx] = make_float2((float)v.x, (float)v.y);
    }
}
// One real value in the arithmetic type (double; double-float hi, lo; float)
__device__ __forceinline__ void put_real(void* q, size_t idx, double v, int prec) {
    if (prec == 0) {
        ((double*)q)[idx] = v;
    } else if (prec == 3) {
        const DF x(v);
        ((float2*)q)[idx] = make_float2(x.hi, x.lo);
    } else {
        ((float*)q)[idx] = (float)v;
    }
}

__global__ void profile_kernel(double M, double a, double rstar_min, double drs, int off, double dth,
                               double rs0, double sig_r, double sig_t, double drs0_dr0,
                               const double* x_int, const double* x_half, SourceDev src,
                               double2* P_int, double2* P_half, double2* dP_int,
                               double2* dP_half, int prec) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int jj = blockIdx.y;
    if (jj >= src.nj) return;
    double th = (src.j_lo + jj + 0.5) * dth;
    // column-major copy for the step kernels, in their arithmetic type
    auto put_q = [&](const void* q, size_t idx, double2 v) { put_cplx(q, idx, v, prec); };
    if (k < src.ni) {
        int i = src.i_lo + k;
        double2* p = &P_int[(size_t)jj * src.ni + k];
        profile_point(M, a, x_int[i], rstar_min + (i + off) * drs, th, rs0, sig_r, sig_t, drs0_dr0,
                      p, &dP_int[(size_t)jj * src.ni + k]);
        put_q(src.Q_int, (size_t)k * src.q_stride + jj, *p);
    }
    if (k < src.nh) {
        int i = src.h_lo + k;
        double2* p = &P_half[(size_t)jj * src.nh + k];
        profile_point(M, a, x_half[i], rstar_min + ((i + off) + 0.5) * drs, th, rs0, sig_r, sig_t,
                      drs0_dr0, p, &dP_half[(size_t)jj * src.nh + k]);
        put_q(src.Q_half, (size_t)k * src.q_stride + jj, *p);
    }
}

// ---------------------------------------------------------------- moving particle
// A particle on a sampled path: the circular-orbit source with the Gaussian centred on
// the particle, factored so that the step kernels only multiply tabulated values,
//   tau_n(i, j) = A e^{-i m phi_p} g_r(r*_i - r*_p) g_th(theta_j - theta_p) Q(i, j)
//   g_r = exp(-dr^2 / (2 sig_r^2)),  g_th = exp(-dth^2 / (2 sig_t^2)),  each 0 beyond 8 sigma
//   Q   = 4 pi (r^2 + a^2 cos^2) Delta / (Sigma^2 r^3) / (2 pi sig_r sig_t)   (static)
// Step n takes sample 2n at the half nodes (Eq. 13) and 2n + 1 at the integer nodes (Eq. 14).
__global__ void prefactor_kernel(double M, double a, double dth, double norm, const double* x_int,
                                 const double* x_half, SourceDev src, int prec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int jj = blockIdx.y;
    if (jj >= src.nj) return;
    const double th = (src.j_lo + jj + 0.5) * dth;
    const double d = sqrt(M * M - a * a);
    const double rp = M + d, rm = M - d;
    double sn, cs;
    sincos(th, &sn, &cs);
    auto pref = [&](double x) {
        const double r = rp + x;
        const double Delta = x * (x + rp - rm);
        const double R = r * r + a * a;
        const double Sig2 = R * R - a * a * Delta * sn * sn;
        return 4.0 * 3.141592653589793238462643 * (r * r + a * a * cs * cs) * Delta /
               (Sig2 * r * r * r) * norm;
    };
    if (k < src.ni)
        put_cplx(src.Q_int, (size_t)k * src.q_stride + jj, make_double2(pref(x_int[src.i_lo + k]), 0.0), prec);
    if (k < src.nh)
        put_cplx(src.Q_half, (size_t)k * src.q_stride + jj, make_double2(pref(x_half[src.h_lo + k]), 0.0), prec);
}

// Block per step (grid-stride): the amplitudes and the radial and angular factors of
// the step's two samples.
__global__ void trajectory_kernel(double M, double a, int m, double rstar_min, double drs, int off,
                                  double dth, double sig_r, double sig_t, const double* traj,
                                  int64_t n_samples, SourceDev src, int prec) {
    const double d = sqrt(M * M - a * a);
    const double rp = M + d, rm = M - d;
    const int nrow = src.nh + src.ni;
    for (int64_t n = blockIdx.x; n < src.n_traj; n += gridDim.x) {
        for (int q = 0; q < 2; ++q) {   // q = 0: sample 2n, half nodes; q = 1: 2n + 1, integer nodes
            const int64_t k = 2 * n + q;
            const bool have = k < n_samples;
            double rs_p = 0.0, th_p = 0.0;
            if (have) {
                const double* smp = traj + 4 * k;
                rs_p = rstar_of_x(M, rp, rm, smp[0] - rp);
                th_p = smp[1];
                if (threadIdx.x == 0) {
                    double sn, cs;
                    sincos((double)m * smp[2], &sn, &cs);
                    ((double2*)src.amp)[2 * n + q] = make_double2(smp[3] * cs, -(smp[3] * sn));
                }
            } else if (threadIdx.x == 0) {
                ((double2*)src.amp)[2 * n + q] = make_double2(0.0, 0.0);
            }
            const int nc = q == 0 ? src.nh : src.ni;
            const int lo = q == 0 ? src.h_lo : src.i_lo;
            void* gr = (char*)src.gr;
            const size_t base = (size_t)n * nrow + (q == 0 ? 0 : src.nh);
            for (int c = threadIdx.x; c < nc; c += blockDim.x) {
                double g = 0.0;
                if (have) {
                    const double rs = rstar_min + (q == 0 ? ((lo + c + off) + 0.5) : (double)(lo + c + off)) * drs;
                    const double dr = rs - rs_p;
                    if (!(fabs(dr) > 8.0 * sig_r)) g = exp(-0.5 * (dr * dr / (sig_r * sig_r)));
                }
                put_real(gr, base + c, g, prec);
            }
            void* gt = (char*)src.gt;
            for (int jj = threadIdx.x; jj < src.nj; jj += blockDim.x) {
                double g = 0.0;
                if (have) {
                    const double dt_ = (src.j_lo + jj + 0.5) * dth - th_p;
                    if (!(fabs(dt_) > 8.0 * sig_t)) g = exp(-0.5 * (dt_ * dt_ / (sig_t * sig_t)));
                }
                put_real(gt, ((size_t)n * 2 + q) * src.nj + jj, g, prec);
            }
        }
    }
}

// 1D tables of the FP32 paths (see RTab2 / ThTab), computed in FP64 and rounded once.
struct RadialVals { double R2, naD, Rd, ctr, cti, ctc, pr, pi, nbb, Ds, nDs, qr, qi, nsdt; };

__device__ RadialVals radial_vals(double M, double a, int s_, int m_, double x, double drs, double sdt) {
    double d = sqrt(M * M - a * a);
    double rp = M + d, rm = M - d;
    double s = (double)s_, m = (double)m_;
    double r = rp + x;
    double Delta = x * (x + rp - rm);
    double R = r * r + a * a;
    RadialVals t;
    t.R2 = R * R;
    t.naD = -(a * a * Delta);
    t.Rd = sdt * R / drs;
    t.ctr = 2.0 * s * (r * Delta - M * (r * r - a * a));
    t.cti = 4.0 * M * a * m * r;
    t.ctc = 2.0 * s * a * Delta;
    t.pr = sdt / drs * (Delta * (6.0 * R / r + 2.0 * r) + 2.0 * R * s * (r - M));
    t.pi = sdt / drs * (2.0 * R * m * a);
    t.nbb = -(sdt / drs * (a * a * Delta * (2.0 * R * (r - M) - 4.0 * r * Delta) * 0.5));
    t.Ds = sdt * Delta;
    t.nDs = -t.Ds;
    t.qr = sdt * (6.0 * Delta * Delta / (r * r) + 6.0 * Delta * (s + 1.0) * (r - M) / r);
    t.qi = sdt * (6.0 * Delta * m * a / r + 4.0 * s * m * a * (r - M));
    t.nsdt = -sdt;
    return t;
}

__device__ float2 pair_f(double h, double i) { return make_float2((float)h, (float)i); }

__global__ void tables_1d_kernel(double M, double a, int s, int m, double drs, double dth,
                                 double dt, int nr, int nth, const double* x_int,
                                 const double* x_half, RTab2* rtab, ThTab* thtab) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nr) {
        // the half node nr-1/2 lies outside the grid: zeros
        const RadialVals h = k < nr - 1 ? radial_vals(M, a, s, m, x_half[k], drs, 0.5 * dt) : RadialVals{};
        const RadialVals i = radial_vals(M, a, s, m, x_int[k], drs, dt);
        RTab2 t;
        t.R2 = pair_f(h.R2, i.R2);
        t.naD = pair_f(h.naD, i.naD);
        t.Rd = pair_f(h.Rd, i.Rd);
        t.ctr = pair_f(h.ctr, i.ctr);
        t.cti = pair_f(h.cti, i.cti);
        t.ctc = pair_f(h.ctc, i.ctc);
        t.pr = pair_f(h.pr, i.pr);
        t.pi = pair_f(h.pi, i.pi);
        t.nbb = pair_f(h.nbb, i.nbb);
        t.Ds = pair_f(h.Ds, i.Ds);
        t.nDs = pair_f(h.nDs, i.nDs);
        t.qr = pair_f(h.qr, i.qr);
        t.qi = pair_f(h.qi, i.qi);
        t.nsdt = pair_f(h.nsdt, i.nsdt);
        t.pad0 = t.pad1 = make_float2(0.f, 0.f);
        rtab[k] = t;
    }
    if (k < nth) {
        double th = (k + 0.5) * dth, sn, cs;
        sincos(th, &sn, &cs);
        double sv = (double)s, mv = (double)m;
        ThTab t;
        t.sin2 = (float)(sn * sn);
        t.cs = (float)cs;
        t.V = (float)((mv + sv * cs) * (mv + sv * cs) / (sn * sn) - sv);
        t.i2 = (float)(1.0 / (dth * dth));
        t.i1 = (float)(cs / sn / (2.0 * dth));
        t.pad0 = t.pad1 = t.pad2 = 0.f;
        thtab[k] = t;
    }
}

void launch_tables_1d(cudaStream_t st, double M, double a, int s, int m, double drs, double dth,
                      double dt, int nr, int nth, const double* x_int, const double* x_half,
                      RTab2* rtab, ThTab* thtab) {
    int n = nr > nth ? nr : nth;
    tables_1d_kernel<<<(n + 127) / 128, 128, 0, st>>>(M, a, s, m, drs, dth, dt, nr, nth, x_int,
                                                      x_half, rtab, thtab);
}

void launch_invert_tortoise(cudaStream_t st, double M, double a, double rstar_min, double drs,
                            int nr, int off, double* x_int, double* x_half) {
    invert_tortoise_kernel<<<(nr + 127) / 128, 128, 0, st>>>(M, a, rstar_min, drs, nr, off, x_int,
                                                              x_half);
}

void launch_coefficients(cudaStream_t st, int prec, double M, double a, int s, int m,
                         double rstar_min, double drs, double dth, double dt, int nr, int nth,
                         int pitch, const double* x_int, const double* x_half, void* coef_h,
                         void* coef_i) {
    dim3 g(nr, (pitch + 127) / 128);
    if (prec == 0)
        coef_kernel<double><<<g, 128, 0, st>>>(M, a, s, m, rstar_min, drs, dth, dt, nr, nth, pitch,
                                               x_int, x_half, (double*)coef_h, (double*)coef_i);
    else if (prec == 3)
        coef_kernel<DF><<<g, 128, 0, st>>>(M, a, s, m, rstar_min, drs, dth, dt, nr, nth, pitch,
                                           x_int, x_half, (DF*)coef_h, (DF*)coef_i);
    else
        coef_kernel<float><<<g, 128, 0, st>>>(M, a, s, m, rstar_min, drs, dth, dt, nr, nth, pitch,
                                              x_int, x_half, (float*)coef_h, (float*)coef_i);
}

void launch_profile(cudaStream_t st, double M, double a, double rstar_min, double drs, int off,
                    double dth, double rs0, double sig_r, double sig_t, double drs0_dr0,
                    const double* x_int, const double* x_half, const SourceDev& src, int prec) {
    dim3 g(((src.ni > src.nh ? src.ni : src.nh) + 127) / 128, src.nj);
    profile_kernel<<<g, 128, 0, st>>>(M, a, rstar_min, drs, off, dth, rs0, sig_r, sig_t, drs0_dr0,
                                      x_int, x_half, src, (double2*)src.P_int,
                                      (double2*)src.P_half, (double2*)src.dP_int,
                                      (double2*)src.dP_half, prec);
}


void launch_trajectory(cudaStream_t st, double M, double a, int m, double rstar_min, double drs,
                       int off, double dth, double sig_r, double sig_t, const double* x_int,
                       const double* x_half, const double* traj, int64_t n_samples,
                       const SourceDev& src, int prec) {
    dim3 g(((src.ni > src.nh ? src.ni : src.nh) + 127) / 128, src.nj);
    prefactor_kernel<<<g, 128, 0, st>>>(M, a, dth, 1.0 / (2.0 * 3.141592653589793238462643 * sig_r * sig_t),
                                        x_int, x_half, src, prec);
    const int64_t blocks = src.n_traj < 4096 ? src.n_traj : 4096;
    trajectory_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 128, 0, st>>>(
        M, a, m, rstar_min, drs, off, dth, sig_r, sig_t, traj, n_samples, src, prec);
}

}  // namespace teuk
