// teuk_step.cu -- the Lax-Wendroff step (Eqs. 13-14) as one fused kernel per step.
//
// Work decomposition: a warp owns a strip of 32 consecutive r* columns (lane L holds
// column i = 30*strip + L) and streams down a chunk of theta rows.  Each lane
// computes the predictor (Eq. 13) at its right half node i+1/2; the left half node
// i-1/2 comes from lane L-1 through a warp shuffle, so lanes 1..30 produce the
// corrector (Eq. 14) for 30 columns per strip.  In theta the warp keeps a 3-row
// register ring of half-node results, so every input row is read from HBM once
// per chunk (plus a 2-row halo at each chunk edge) and nothing goes through shared
// memory.  The angular ghost rows of the pole boundary condition (Sec. 2.2) are
// mirror images of row 0 / row n_theta-1 with sign +1 (even |m|) or -1 (odd |m|),
// applied to the state for the predictor and to the half-node results for the
// corrector.
//
// Arithmetic, in terms of differences so that the compensated FP32 state keeps
// its accuracy (a difference of two (hi, c) pairs is formed as
// (hi_a - hi_b) - (c_a - c_b) before anything cancels):
//   predictor at (i+1/2, j), with Fb = (Phi_i + Phi_{i+1})/2, dF = Phi_{i+1} - Phi_i,
//   Dp(j) = Fb(j+1) - Fb(j) and the same for Pi:
//     dh_Phi = -g dF + (dt/2) Pb
//     dh_Pi  =  g dPi + E1 Pb + E2 dF + ep Dp(j) - em Dp(j-1) + E3 Fb + (dt/2) tau(t_n)
//   corrector at (i, j) from the half nodes R = i+1/2, L = i-1/2:
//     h_R - h_L = (dF_R + dF_L)/2 + dh_R - dh_L,  u~ = (Fb_R + Fb_L)/2 + (dh_R + dh_L)/2,
//     Delta Phi = -g d(h_Phi) + dt Pi~
//     Delta Pi  =  g d(h_Pi) + E1 Pi~ + E2 d(h_Phi) + ep D+ - em D- + E3 Phi~ + dt tau(t_n+dt/2)
//     u^{n+1} = u^n + Delta   (Kahan-compensated for the FP32_KAHAN state)
// with the scaled coefficients g, E1, E2, ep, em, E3 of teuk_setup.cu (the two
// sub-steps differ only by the factor 1/2 versus 1 of dt).  This is Eqs. (13)-(14)
// with S_Pi = -c_t Pi + P* Phi_* + w Theta[Phi] + q Phi + tau, rearranged, not
// approximated.
#include "teuk_internal.cuh"
#include "teuk_step_common.cuh"

namespace teuk {

template <class P>
__global__ void __launch_bounds__(128) step_kernel(InstDev d, int64_t step, int bin, int chunk) {
    using T = typename P::T;
    using C = Cx<T>;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nstrip = (d.nr - 2 + 29) / 30;
    const int nck = (d.nth + chunk - 1) / chunk;
    if (gw >= nstrip * nck) return;  // whole warps only
    const int strip = gw % nstrip, ck = gw / nstrip;
    const int i = 30 * strip + lane;
    const bool col_ok = i < d.nr;
    const bool half_ok = lane < 31 && i + 1 < d.nr;
    const bool out_ok = lane >= 1 && lane <= 30 && i <= d.nr - 2;
    const bool bnd = (i == 0 || i == d.nr - 1) && (lane <= 30);
    const int j0 = ck * chunk, j1 = min(d.nth, j0 + chunk);
    const int nth = d.nth, pitch = d.pitch;
    const size_t pl = plane_elems(d);
    const T* ch = (const T*)d.coef_h;
    const T* ci = (const T*)d.coef_i;
    const T g = (T)d.ghost;
    const T hdt = (T)(0.5 * d.dt), fdt = (T)d.dt;
    const int ex_strip = d.i_e >= 1 ? (d.i_e - 1) / 30 : 0;
    const bool ex_warp = strip == ex_strip;

    // source factors of this step: (dt/2) A_n e^{-i(omega t_n + phase0)} and
    // dt A_n e^{-i(omega (t_n + dt/2) + phase0)}, FP64
    double2 sp_fac = make_double2(0.0, 0.0), sc_fac = make_double2(0.0, 0.0);
    if (d.src.on) source_factors(d, step, sp_fac, sc_fac);

    const Planes<P> in = Planes<P>::of(d, bin), out = Planes<P>::of(d, 1 - bin);

    NodeV<P> prev = NodeV<P>::zero();
    Half<T> pend;           // Fb, Pb, dF, dP of the previous loaded row
    C dp_prev = C::zero();  // Dp of row (previous loaded row - 1)
    CRing<T> ring;          // corrector inputs of rows jc-1, jc, jc+1
    int ring_n = 0;         // rows pushed so far
    int ring_top = -3;      // row index of ring.c

    const int jl_begin = max(j0 - 2, -1), jl_end = min(j1 + 1, nth);
    const int jp_lo = max(j0 - 1, 0), jp_hi = min(j1, nth - 1);

    for (int jl = jl_begin; jl <= jl_end; ++jl) {
        // ---- load row jl of the own column (mirror rows outside [0, nth)) ----
        const int jr = jl < 0 ? 0 : (jl >= nth ? nth - 1 : jl);
        NodeV<P> own = col_ok ? in.load((size_t)jr * pitch + i) : NodeV<P>::zero();
        if (jl < 0 || jl >= nth) own.scale(g);
        const NodeV<P> nb = own.shfl_down();
        Half<T> cur = half_prep<P>(own, nb);
        C dp_cur = C::zero();
        if (jl > jl_begin) {
            // Dp(jl-1) = Fb(jl) - Fb(jl-1), from the columns' own theta differences
            C delta = own.dphi(prev);
            C delta_n = shfl_down_c(delta);
            dp_cur = C::half_sum(delta, delta_n);
        }
        prev = own;

        // ---- predictor at jp = jl - 1 ----
        const int jp = jl - 1;
        if (jl > jl_begin && jp >= jp_lo && jp <= jp_hi) {
            T cf[kNCoef];
            load_coefs(ch, pl, (size_t)jp * pitch + i, half_ok, cf);
            C src = C::zero();
            if (d.src.on) src = source_half<T>(d.src, sp_fac, i, jp);
            HalfRec<T> rec = predictor<T>(pend, dp_cur, dp_prev, cf, hdt, src);
            CRow<T> row = combine_lr<T>(rec);
            if (jp == 0) {  // ghost row -1 of the half-node results
                CRow<T> gr = row.mirror(g);
                gr.DpS = C::half_sum(dp_prev, shfl_up_c(dp_prev));
                ring.push(gr);
                ++ring_n;
                ring_top = -1;
            }
            ring.push(row);
            ++ring_n;
            ring_top = jp;
            if (ring_n >= 3 && ring_top - 1 >= j0 && ring_top - 1 < j1)
                corrector<P>(d, in, out, ring, ring_top - 1, i, out_ok, bnd, ex_warp, ci, pl,
                             fdt, sc_fac, step);
            if (jp == nth - 1) {  // ghost row nth
                CRow<T> gr = row.mirror(g);
                ring.push(gr);
                ++ring_n;
                ring_top = nth;
                if (ring_n >= 3 && nth - 1 >= j0 && nth - 1 < j1)
                    corrector<P>(d, in, out, ring, nth - 1, i, out_ok, bnd, ex_warp, ci, pl, fdt,
                                 sc_fac, step);
            }
        }
        pend = cur;
        dp_prev = dp_cur;
    }
}

// Waveform record of the state in buffer bin (time level `step`): one thread per row.
template <class P>
__global__ void extract_kernel(InstDev d, int64_t step, int bin) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.nth) return;
    const Planes<P> in = Planes<P>::of(d, bin);
    size_t o = (size_t)j * d.pitch + d.i_e;
    double2 a = in.load(o).phi64(), b = in.load(o + 1).phi64();
    double f = d.f_e;
    double2 w = make_double2((1.0 - f) * a.x + f * b.x, (1.0 - f) * a.y + f * b.y);
    d.wave[(size_t)(step % d.wave_cap) * d.nth + j] = w;
    if (!isfinite(w.x) || !isfinite(w.y)) atomicOr(d.status, (unsigned)ST_NONFINITE);
}

void launch_step(cudaStream_t st, const InstDev& d, int64_t step, int bin, int chunk) {
    int nstrip = (d.nr - 2 + 29) / 30;
    int nck = (d.nth + chunk - 1) / chunk;
    int64_t warps = (int64_t)nstrip * nck;
    int blocks = (int)((warps * 32 + 127) / 128);
    if (d.prec == 0) step_kernel<P64><<<blocks, 128, 0, st>>>(d, step, bin, chunk);
    else if (d.prec == 1) step_kernel<P32><<<blocks, 128, 0, st>>>(d, step, bin, chunk);
    else step_kernel<PK><<<blocks, 128, 0, st>>>(d, step, bin, chunk);
}

void launch_extract(cudaStream_t st, const InstDev& d, int64_t step, int bin) {
    int blocks = (d.nth + 127) / 128;
    if (d.prec == 0) extract_kernel<P64><<<blocks, 128, 0, st>>>(d, step, bin);
    else if (d.prec == 1) extract_kernel<P32><<<blocks, 128, 0, st>>>(d, step, bin);
    else extract_kernel<PK><<<blocks, 128, 0, st>>>(d, step, bin);
}

}  // namespace teuk
