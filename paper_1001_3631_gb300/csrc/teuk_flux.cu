// teuk_flux.cu -- energy, linear momentum and angular momentum about the spin axis
// carried off by the field of several modes (the recoil of Sec. 2.2), from the modes'
// waveform records at the extraction radius.
//
// Per mode i and theta row j the records give r psi_4 = Phi e^{i m phi~} F_j with the
// Kerr factor F_j = (r / (r - i a cos theta_j))^4 (psi_4 = rho^4 Psi for s = -2,
// Psi = e^{i m phi~} r^3 Phi of Eq. 4) and phi~ = phi + shift (Eq. 3 at the radius).
// With N = int r psi_4 dt and H = int N dt (trapezoid rule from the first record),
// the azimuth integrals of the flux formulas reduce by the orthogonality of e^{i m phi}:
//   dE/dt       = 1/2 sum_i sum_j w_j |N_ij|^2                       (w_j = sin th_j dth)
//   dPz/dt      = 1/2 sum_i sum_j w_j cos th_j |N_ij|^2
//   dPx + i dPy = 1/2 sum_i sum_j w_j sin th_j N_ij conj(N_i'j)      (m_i' = m_i + 1)
//   dJz/dt      = 1/2 sum_i m_i sum_j w_j Im(conj(N_ij) H_ij)
// and E, P, Jz are trapezoid integrals of the rates from the first record.
//
// The factor F_ij = (r / (r - i a cos theta_j))^4 e^{i m_i shift} is constant in time, so
// the scans integrate the records themselves (N = F Nw, H = F Hw with Nw = int W dt,
// Hw = int Nw dt) and F enters the sums once per entry: w_j |F|^2 for E, Pz and Jz,
// w_j sin th_j F_i conj(F_i') for the x-y momentum (formed with the chunk starts).
// The time integrals are scans along the records.  They run in chunks of Lc records:
// one pass integrates every chunk from zero (its totals), a second carries the totals
// from chunk to chunk (N and H at each chunk's start; H gains n dt N_start over a
// chunk of n steps), a third integrates every chunk again from its start, a block per
// (chunk, group of rows of every mode), and sums each record's terms over the block
// in a fixed order (each term by one warp: per lane over the warps, then a shuffle
// tree); the last adds the groups' sums of each record in order and scans the rates
// into the totals, one block per quantity.  All arithmetic is FP64, and the results do
// not depend on the scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "teuk_aux.cuh"

namespace teuk {
namespace {

constexpr double kPi = 3.141592653589793238462643;

__device__ __forceinline__ double2 cmul(double2 x, double2 y) {
    return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}
__device__ __forceinline__ double2 cadd(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }
__device__ __forceinline__ double2 cscale(double s, double2 x) { return make_double2(s * x.x, s * x.y); }

// F_ij = (r / (r - i a cos th_j))^4 e^{i m_i shift}: turns mode i's record at row j into
// r psi_4 without its e^{i m phi}
__device__ double2 entry_factor(const FluxDev& f, int i, double cth) {
    const double den = f.r * f.r + f.a * f.a * cth * cth;
    double2 z = make_double2(f.r * f.r / den, f.r * f.a * cth / den);   // r / (r - i a c)
    z = cmul(z, z);
    z = cmul(z, z);
    double sn, cs;
    sincos((double)f.modes[i].m * f.shift, &sn, &cs);
    return cmul(z, make_double2(cs, sn));
}

__device__ __forceinline__ double2 record(const FluxDev& f, const ModeRing& q, int j, int64_t k) {
    return q.wave[(size_t)((f.first + k) % q.cap) * f.nth + j];
}

// chunk c advances the records s_c -> e_c (s_0 = 0, s_c = c Lc - 1, e_c = min((c+1) Lc, R) - 1)
__device__ __forceinline__ int64_t chunk_start(const FluxDev& f, int c) {
    return c == 0 ? 0 : (int64_t)c * f.Lc - 1;
}
__device__ __forceinline__ int64_t chunk_end(const FluxDev& f, int c) {
    const int64_t e = (int64_t)(c + 1) * f.Lc;
    return (e < f.R ? e : f.R) - 1;
}

// Pass 1: every chunk's Nw and Hw integrated from zero at its start record.
__global__ void flux_chunk_totals_kernel(FluxDev f, double2* totN, double2* totH) {
    const int E = f.K * f.nth;
    const int64_t total = (int64_t)f.n_chunks * E;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx % E), c = (int)(idx / E);
        const int i = e / f.nth, j = e % f.nth;
        const ModeRing q = f.modes[i];
        const double hdt = 0.5 * f.dt;
        double2 N = make_double2(0.0, 0.0), H = N;
        double2 Cp = record(f, q, j, chunk_start(f, c));
        const int64_t k1 = chunk_end(f, c);
        for (int64_t k = chunk_start(f, c) + 1; k <= k1; ++k) {
            const double2 Cc = record(f, q, j, k);
            const double2 Nn = cadd(N, cscale(hdt, cadd(Cp, Cc)));
            H = cadd(H, cscale(hdt, cadd(N, Nn)));
            N = Nn;
            Cp = Cc;
        }
        totN[idx] = N;
        totH[idx] = H;
    }
}

// Pass 2: Nw and Hw at every chunk's start record, chunk after chunk; also each entry's
// weights: g = (w_j |F|^2, w_j cos th_j |F|^2, m_i w_j |F|^2) and gp = w_j sin th_j
// F_i conj(F_i') (zero without a partner).
__global__ void flux_chunk_starts_kernel(FluxDev f, const int* __restrict__ partner,
                                         const double2* __restrict__ totN, const double2* __restrict__ totH,
                                         double2* __restrict__ stN, double2* __restrict__ stH,
                                         FluxWeights* __restrict__ g, double2* __restrict__ gp) {
    const int E = f.K * f.nth;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const int i = e / f.nth, j = e % f.nth;
        const double dth = kPi / (double)f.nth;
        double sn, cs;
        sincos(((double)j + 0.5) * dth, &sn, &cs);
        const double w = sn * dth;
        const double2 F = entry_factor(f, i, cs);
        const double a2 = w * (F.x * F.x + F.y * F.y);
        g[e] = FluxWeights{a2, a2 * cs, (double)f.modes[i].m * a2, 0.0};
        double2 x = make_double2(0.0, 0.0);
        const int ip = partner[i];
        if (ip >= 0) {
            const double2 Fp = entry_factor(f, ip, cs);
            x = cscale(w * sn, cmul(F, make_double2(Fp.x, -Fp.y)));
        }
        gp[e] = x;
        double2 N = make_double2(0.0, 0.0), H = N;
        stN[e] = N;
        stH[e] = H;
        // the chain over chunks is sequential; its loads are not, so they go out 8 at a time
        constexpr int U = 8;
        for (int c0 = 0; c0 + 1 < f.n_chunks; c0 += U) {
            double2 tn[U], th[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c0 + u + 1 < f.n_chunks) {
                    tn[u] = totN[(size_t)(c0 + u) * E + e];
                    th[u] = totH[(size_t)(c0 + u) * E + e];
                }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c0 + u + 1 < f.n_chunks) {
                    const int c = c0 + u;
                    const double n = (double)(chunk_end(f, c) - chunk_start(f, c));
                    H = cadd(cadd(H, cscale(n * f.dt, N)), th[u]);
                    N = cadd(N, tn[u]);
                    stN[(size_t)(c + 1) * E + e] = N;
                    stH[(size_t)(c + 1) * E + e] = H;
                }
        }
    }
}

// Pass 3: block (b, c): the rows [b RB, b RB + RB) of every mode over the records of
// chunk c, K RB threads rounded up to whole warps (at most 256); thread t = i RB + jj is
// mode i at row j = b RB + jj (mode i's partner, mode m_i + 1, is the thread of the same
// row in its own mode's group).  Record after record: Nw and Hw advanced from the
// chunk's start, Nw published in shared memory, the thread's five terms (the partner's
// Nw read there) written to one of two term buffers, then warp r sums term r (warp
// r mod the block's warps when it has fewer than five): lane l adds the terms of threads
// l, l + 32, ... in order, then a shuffle tree across the lanes, into part[k][b][r].
// The other warps go on to the next record meanwhile (two buffers and two barriers a
// record keep the reads ahead of the next writes).
// Record 0 belongs to chunk 0 and is not advanced.
constexpr int kSumsMaxThreads = 256;

__global__ void __launch_bounds__(kSumsMaxThreads) flux_sums_kernel(FluxDev f, const int* __restrict__ partner,
                                                                    const double2* __restrict__ stN,
                                                                    const double2* __restrict__ stH,
                                                                    const FluxWeights* __restrict__ g,
                                                                    const double2* __restrict__ gp,
                                                                    double* __restrict__ part) {
    __shared__ double2 sN[kSumsMaxThreads];
    __shared__ double sT[2][5][kSumsMaxThreads];
    const int b = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    const int E = f.K * f.nth;
    const int i = t / f.RB, jj = t % f.RB, j = b * f.RB + jj;
    // threads past K RB (the block is whole warps) and rows past the last take no part
    const bool ok = i < f.K && j < f.nth;
    const int e = i * f.nth + j;
    const int ip = ok ? partner[i] : -1;
    const int tp = ip >= 0 ? ip * f.RB + jj : -1;
    const ModeRing q = f.modes[ok ? i : 0];
    const double2 z = make_double2(0.0, 0.0);
    const FluxWeights w = ok ? g[e] : FluxWeights{0.0, 0.0, 0.0, 0.0};
    const double2 p = ok ? gp[e] : z;
    double2 N = ok ? stN[(size_t)c * E + e] : z, H = ok ? stH[(size_t)c * E + e] : z;
    const int64_t ks = chunk_start(f, c), k1 = chunk_end(f, c);
    double2 Cp = ok ? record(f, q, j, ks) : z;
    const double hdt = 0.5 * f.dt;
    const int lane = t & 31, nw = blockDim.x >> 5;
    int buf = 0;
    for (int64_t k = c == 0 ? 0 : ks + 1; k <= k1; ++k, buf ^= 1) {
        if (k > ks) {
            const double2 Cc = ok ? record(f, q, j, k) : z;
            const double2 Nn = cadd(N, cscale(hdt, cadd(Cp, Cc)));
            H = cadd(H, cscale(hdt, cadd(N, Nn)));
            N = Nn;
            Cp = Cc;
        }
        sN[t] = N;
        __syncthreads();
        const double n2 = N.x * N.x + N.y * N.y;
        double x1 = 0.0, x2 = 0.0;
        if (tp >= 0) {
            const double2 u = sN[tp];             // N conj(N')
            const double2 x = make_double2(N.x * u.x + N.y * u.y, N.y * u.x - N.x * u.y);
            x1 = p.x * x.x - p.y * x.y;
            x2 = p.x * x.y + p.y * x.x;
        }
        sT[buf][0][t] = w.e * n2;
        sT[buf][1][t] = x1;
        sT[buf][2][t] = x2;
        sT[buf][3][t] = w.z * n2;
        sT[buf][4][t] = w.jz * (N.x * H.y - N.y * H.x);   // Im(conj(N) H)
        __syncthreads();
        for (int r = t >> 5; r < 5; r += nw) {   // warp r sums term r
            double acc = 0.0;
            for (int v = 0; v < nw; ++v) acc += sT[buf][r][lane + 32 * v];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) part[((size_t)k * gridDim.x + b) * 5 + r] = acc;
        }
    }
}

constexpr int kScanThreads = 1024;

// rate q of record k: half the sum of the row groups' sums, groups in order
__device__ __forceinline__ double rate_of(const double* part, int n_rg, int64_t k, int q) {
    double acc = 0.0;
    for (int b = 0; b < n_rg; ++b) acc += part[((size_t)k * n_rg + b) * 5 + q];
    return 0.5 * acc;
}

// Pass 4: block q scans the rate q into its total (trapezoid from the first record) and
// writes out[k][q] = rate, out[k][5 + q] = total.
__global__ void __launch_bounds__(kScanThreads) flux_totals_kernel(int64_t R, int n_rg, double dt,
                                                                   const double* __restrict__ part,
                                                                   double* __restrict__ out) {
    __shared__ double wsum[kScanThreads / 32];
    __shared__ double rs[kScanThreads + 1];    // the tile's rates after the previous tile's last
    const int q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double carry = 0.0;
    if (threadIdx.x == 0) rs[kScanThreads] = 0.0;
    for (int64_t base = 0; base < R; base += kScanThreads) {
        const int64_t k = base + threadIdx.x;
        const double r = k < R ? rate_of(part, n_rg, k, q) : 0.0;
        __syncthreads();                       // the previous tile is done with rs
        if (threadIdx.x == 0) rs[0] = rs[kScanThreads];
        __syncthreads();
        rs[threadIdx.x + 1] = r;
        __syncthreads();
        const double inc = (k < R && k > 0) ? 0.5 * dt * (rs[threadIdx.x] + r) : 0.0;
        // inclusive scan: within the warp, then over the warps' sums
        double x = inc;
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            double v = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const double before = warp > 0 ? wsum[warp - 1] : 0.0;
        if (k < R) {
            out[k * 10 + q] = r;
            out[k * 10 + 5 + q] = carry + (before + x);
        }
        carry += wsum[kScanThreads / 32 - 1];
    }
}

unsigned grid_of(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int launch_radiated_flux(cudaStream_t st, const FluxDev& f, const FluxScratch& s) {
    const int E = f.K * f.nth;
    int launches = 0;
    if (f.n_chunks > 1) {
        FluxDev g = f;
        g.n_chunks = f.n_chunks - 1;      // the last chunk's totals are not needed
        flux_chunk_totals_kernel<<<grid_of((int64_t)g.n_chunks * E, 256), 256, 0, st>>>(g, s.totN, s.totH);
        ++launches;
    }
    flux_chunk_starts_kernel<<<grid_of(E, 128), 128, 0, st>>>(f, s.partner, s.totN, s.totH, s.stN,
                                                              s.stH, s.g, s.gp);
    const int threads = (f.K * f.RB + 31) / 32 * 32;
    flux_sums_kernel<<<dim3((unsigned)f.n_rg, (unsigned)f.n_chunks), threads, 0, st>>>(
        f, s.partner, s.stN, s.stH, s.g, s.gp, s.part);
    flux_totals_kernel<<<5, kScanThreads, 0, st>>>(f.R, f.n_rg, f.dt, s.part, s.out);
    return launches + 3;
}

}  // namespace teuk
