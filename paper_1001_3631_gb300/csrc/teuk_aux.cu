// teuk_aux.cu -- small kernels around the time step: conversion between the host
// u-layout and the internal planes, the finiteness scan, the sin(theta)-weighted
// theta sum of the waveform records, and the sum of the records over modes.
#include "teuk_aux.cuh"
#include "teuk_internal.cuh"
#include "teuk_step_common.cuh"

namespace teuk {

// u-layout [4][nth][nr] (Phi_R, Phi_I, Pi_R, Pi_I) -> planes of buffer b.  The
// compensated state is split as hi = fl32(v), c = fl32(hi - v), so hi - c = v to
// about 2^-48 relative; the double-float state as hi = fl32(v), lo = fl32(v - hi).
template <class P>
__global__ void import_state_kernel(InstDev d, int b, const double* u) {
    int j = blockIdx.y * blockDim.x + threadIdx.x;   // theta row
    int i = blockIdx.x;                              // r* column
    if (i >= d.nr || j >= d.nth) return;
    size_t np = (size_t)d.nr * d.nth, q = (size_t)j * d.nr + i, o = node_index(d, i, j);
    double v[4] = {u[q], u[np + q], u[2 * np + q], u[3 * np + q]};
    if constexpr (P::kind == kDF) {
        DF h[4];
        for (int k = 0; k < 4; ++k) h[k] = DF(v[k]);
        ((float4*)d.buf[b][0])[o] = make_float4(h[0].hi, h[1].hi, h[2].hi, h[3].hi);
        ((float4*)d.buf[b][1])[o] = make_float4(h[0].lo, h[1].lo, h[2].lo, h[3].lo);
    } else if constexpr (P::kind == kFP64) {
        ((double2*)d.buf[b][0])[o] = make_double2(v[0], v[1]);
        ((double2*)d.buf[b][1])[o] = make_double2(v[2], v[3]);
    } else if constexpr (!P::kahan) {
        ((float4*)d.buf[b][0])[o] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    } else {
        float h[4], c[4];
        for (int k = 0; k < 4; ++k) {
            h[k] = (float)v[k];
            c[k] = (float)((double)h[k] - v[k]);
        }
        ((float4*)d.buf[b][0])[o] = make_float4(h[0], h[1], h[2], h[3]);
        ((float4*)d.buf[b][1])[o] = make_float4(c[0], c[1], c[2], c[3]);
    }
}

template <class P>
__global__ void export_state_kernel(InstDev d, int b, double* u) {
    int j = blockIdx.y * blockDim.x + threadIdx.x;   // theta row
    int i = blockIdx.x;                              // r* column
    if (i >= d.nr || j >= d.nth) return;
    size_t np = (size_t)d.nr * d.nth, q = (size_t)j * d.nr + i, o = node_index(d, i, j);
    NodeV<P> n = Planes<P>::of(d, b).load(o);
    double v[4];
    n.v64(v);
    u[q] = v[0]; u[np + q] = v[1]; u[2 * np + q] = v[2]; u[3 * np + q] = v[3];
}

// Sets ST_NONFINITE if any state value of buffer b is NaN or infinite.
template <class P>
__global__ void scan_finite_kernel(InstDev d, int b) {
    int j = blockIdx.y * blockDim.x + threadIdx.x;   // theta row
    int i = blockIdx.x;                              // r* column
    if (i >= d.nr || j >= d.nth) return;
    NodeV<P> n = Planes<P>::of(d, b).load(node_index(d, i, j));
    double v[4];
    n.v64(v);
    bool ok = isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]);
    if constexpr (P::kahan)
        ok = ok && isfinite(n.Fc.re) && isfinite(n.Fc.im) && isfinite(n.Pc.re) && isfinite(n.Pc.im);
    if (!ok) atomicOr(d.status, (unsigned)ST_NONFINITE);
}

// out[k] = sum_j W[level0 + k][j] sin(theta_j) dtheta, j ascending, FP64.
__global__ void wave_sum_kernel(const double2* wave, int64_t cap, int nth, double dth,
                                int64_t level0, int64_t k_count, double2* out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= k_count) return;
    const double2* w = wave + (size_t)((level0 + k) % cap) * nth;
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < nth; ++j) {
        double sn = sin((j + 0.5) * dth) * dth;
        sr += w[j].x * sn;
        si += w[j].y * sn;
    }
    out[k] = make_double2(sr, si);
}

// Zero both buffers' planes (padding included).
__global__ void zero_kernel(double* p, size_t n) {
    size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; k < n; k += stride) p[k] = 0.0;
}

void launch_import_state(cudaStream_t st, const InstDev& d, int bin, const double* u) {
    dim3 g(d.nr, (d.nth + 127) / 128);
    if (d.prec == 0) import_state_kernel<P64><<<g, 128, 0, st>>>(d, bin, u);
    else if (d.prec == 1) import_state_kernel<P32><<<g, 128, 0, st>>>(d, bin, u);
    else if (d.prec == 3) import_state_kernel<PD><<<g, 128, 0, st>>>(d, bin, u);
    else import_state_kernel<PK><<<g, 128, 0, st>>>(d, bin, u);
}

void launch_export_state(cudaStream_t st, const InstDev& d, int bin, double* u) {
    dim3 g(d.nr, (d.nth + 127) / 128);
    if (d.prec == 0) export_state_kernel<P64><<<g, 128, 0, st>>>(d, bin, u);
    else if (d.prec == 1) export_state_kernel<P32><<<g, 128, 0, st>>>(d, bin, u);
    else if (d.prec == 3) export_state_kernel<PD><<<g, 128, 0, st>>>(d, bin, u);
    else export_state_kernel<PK><<<g, 128, 0, st>>>(d, bin, u);
}

void launch_scan_finite(cudaStream_t st, const InstDev& d, int bin) {
    dim3 g(d.nr, (d.nth + 127) / 128);
    if (d.prec == 0) scan_finite_kernel<P64><<<g, 128, 0, st>>>(d, bin);
    else if (d.prec == 1) scan_finite_kernel<P32><<<g, 128, 0, st>>>(d, bin);
    else if (d.prec == 3) scan_finite_kernel<PD><<<g, 128, 0, st>>>(d, bin);
    else scan_finite_kernel<PK><<<g, 128, 0, st>>>(d, bin);
}

void launch_wave_sum(cudaStream_t st, const double2* wave, int64_t cap, int nth, double dth,
                     int64_t level0, int64_t k_count, double2* out) {
    wave_sum_kernel<<<(unsigned)((k_count + 127) / 128), 128, 0, st>>>(wave, cap, nth, dth, level0,
                                                                     k_count, out);
}

// Thread per (record k, row j, azimuth l), grid-stride; the modes are added in order.
__global__ void mode_sum_kernel(const ModeRing* modes, int n_modes, int nth, const double* phi,
                                int n_phi, int64_t first, int64_t n_rec, double r3, double shift,
                                double2* out) {
    const int64_t total = n_rec * nth * n_phi;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx % n_phi);
        const int64_t t = idx / n_phi;
        const int j = (int)(t % nth);
        const int64_t k = t / nth;
        const double ph = phi[l] + shift;
        double re = 0.0, im = 0.0;
        for (int i = 0; i < n_modes; ++i) {
            const ModeRing q = modes[i];
            const double2 w = q.wave[(size_t)((first + k) % q.cap) * nth + j];
            double sn, cs;
            sincos((double)q.m * ph, &sn, &cs);
            re += cs * w.x - sn * w.y;
            im += cs * w.y + sn * w.x;
        }
        out[idx] = make_double2(r3 * re, r3 * im);
    }
}

void launch_mode_sum(cudaStream_t st, const ModeRing* modes, int n_modes, int nth,
                     const double* phi, int n_phi, int64_t first, int64_t n_rec, double r3,
                     double shift, double2* out) {
    const int64_t total = n_rec * nth * n_phi;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    mode_sum_kernel<<<(unsigned)blocks, 256, 0, st>>>(modes, n_modes, nth, phi, n_phi, first,
                                                      n_rec, r3, shift, out);
}

// (checked builds) the bounds check of an index one past the end of the state plane; the
// index is only tested, never addressed
__global__ void check_selftest_kernel(InstDev d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool in = TK_IN(d.status, plane_elems(d), plane_elems(d));
        (void)in;
    }
}

void launch_check_selftest(cudaStream_t st, const InstDev& d) {
    check_selftest_kernel<<<1, 32, 0, st>>>(d);
}

}  // namespace teuk
