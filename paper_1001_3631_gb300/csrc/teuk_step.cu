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

// One work item: the strip `strip` (columns 30*strip .. 30*strip+31) and the theta
// chunk `ck` (rows ck*chunk .. ) of one step, executed by one whole warp.
template <class P>
__device__ __forceinline__ void step_item(const InstDev& d, int64_t step, int bin, int chunk,
                                          int strip, int ck) {
    using T = typename P::T;
    using C = Cx<T>;
    const int lane = threadIdx.x & 31;
    const int i = 30 * strip + lane;
    const bool col_ok = i < d.nr;
    const bool half_ok = lane < 31 && i + 1 < d.nr;
    const bool out_ok = lane >= 1 && lane <= 30 && i <= d.nr - 2;
    const bool bnd = (i == 0 || i == d.nr - 1) && (lane <= 30);
    const int j0 = ck * chunk, j1 = min(d.nth, j0 + chunk);
    const int nth = d.nth, pitch = d.pitch;
    const T g = (T)d.ghost;
    const T hdt = (T)(0.5 * d.dt), fdt = (T)d.dt;
    const int ex_strip = d.i_e >= 1 ? (d.i_e - 1) / 30 : 0;
    const bool ex_warp = strip == ex_strip;

    // source factors of this step: (dt/2) A_n e^{-i(omega t_n + phase0)} and
    // dt A_n e^{-i(omega (t_n + dt/2) + phase0)}, FP64
    // only warps whose columns and rows meet the source window need them
    const int c_lo = 30 * strip, c_hi = 30 * strip + 31, r_lo = j0 - 1, r_hi = j1;
    const SourceDev& sw = d.src;
    const bool src_warp = sw.on && r_lo < sw.j_lo + sw.nj && r_hi >= sw.j_lo &&
                          ((c_lo < sw.i_lo + sw.ni && c_hi >= sw.i_lo) ||
                           (c_lo < sw.h_lo + sw.nh && c_hi >= sw.h_lo));
    double2 sp_fac = make_double2(0.0, 0.0), sc_fac = make_double2(0.0, 0.0);
    if (src_warp) source_factors(d, step, sp_fac, sc_fac);

    const Planes<P> in = Planes<P>::of(d, bin), out = Planes<P>::of(d, 1 - bin);
    ColTab<P> colh, coli;  // radial coefficient tables of this lane's column (FP32 paths)
    colh.load(d.rtab_h, i, half_ok);
    coli.load(d.rtab_i, i, col_ok);

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
            get_coefs<P>(d, colh, true, i, jp, half_ok, cf);
            C src = C::zero();
            if (src_warp) src = source_half<T>(d.src, sp_fac, i, jp);
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
                corrector<P>(d, in, out, ring, ring_top - 1, i, out_ok, bnd, ex_warp, src_warp,
                             coli, fdt, sc_fac, step);
            if (jp == nth - 1) {  // ghost row nth
                CRow<T> gr = row.mirror(g);
                ring.push(gr);
                ++ring_n;
                ring_top = nth;
                if (ring_n >= 3 && nth - 1 >= j0 && nth - 1 < j1)
                    corrector<P>(d, in, out, ring, nth - 1, i, out_ok, bnd, ex_warp, src_warp,
                                 coli, fdt, sc_fac, step);
            }
        }
        pend = cur;
        dp_prev = dp_cur;
    }
}

template <class P>
__global__ void __launch_bounds__(128) step_kernel(InstDev d, int64_t step, int bin, int chunk) {
    const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nstrip = (d.nr - 2 + 29) / 30;
    const int nck = (d.nth + chunk - 1) / chunk;
    if (gw >= nstrip * nck) return;  // whole warps only
    step_item<P>(d, step, bin, chunk, gw % nstrip, gw / nstrip);
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

// ---------------------------------------------------------------- batched path
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until the items of the 3x3 neighbourhood (strips strip-1..strip+1, chunks
// ck-1..ck+1) have completed relative step s-1.  That covers what this item reads
// (halo of one column and two rows) and what it overwrites (the buffer the
// neighbours of step s-1 read).  Lanes 0..8 each poll one neighbour with acquire
// loads; the wait gives up after spin_limit polls.  Returns false on give-up or abort.
__device__ bool wait_neighbours(const BatchDev& b, const int* fl, int nstrip, int nck, int strip,
                                int ck, int64_t s) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < 9) {
        int st = strip + lane % 3 - 1, c = ck + lane / 3 - 1;
        if (st >= 0 && st < nstrip && c >= 0 && c < nck) {
            const int* f = fl + (size_t)c * nstrip + st;
            long long it = 0;
            while (ld_acquire(f) < (int)s) {
                if (++it > b.spin_limit || *(volatile int*)b.abort) { ok = false; break; }
                __nanosleep(64);
            }
        }
    }
    ok = __all_sync(kFull, ok);
    __threadfence();
    return ok;
}

template <class P>
__global__ void __launch_bounds__(128) batched_step_kernel(BatchDev b) {
    const int lane = threadIdx.x & 31;
    const int64_t nsteps = *b.n_steps;
    const int64_t total = b.items_per_step * nsteps;
    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(b.counter, 1ull);
        g = __shfl_sync(kFull, g, 0);
        if ((int64_t)g >= total) return;
        if (*(volatile int*)b.abort) return;
        const int64_t s = (int64_t)g / b.items_per_step, r = (int64_t)g % b.items_per_step;
        int lo = 0, hi = b.n_inst - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (b.item_base[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const int k = lo;
        const int64_t local = r - b.item_base[k];
        const InstDev& d = b.inst[k];
        const int nstrip = b.nstrip[k], chunk = b.chunk[k];
        const int nck = (d.nth + chunk - 1) / chunk;
        const int ck = (int)(local / nstrip), strip = (int)(local % nstrip);
        int* fl = b.flags + b.item_base[k];
        if (s > 0 && !wait_neighbours(b, fl, nstrip, nck, strip, ck, s)) {
            if (lane == 0) {
                atomicOr(b.status, (unsigned)ST_TIMEOUT);
                atomicExch(b.abort, 1);
            }
            return;
        }
        step_item<P>(d, b.base_step[k] + s, (int)((b.base_bin[k] + s) & 1), chunk, strip, ck);
        __threadfence();
        __syncwarp();
        if (lane == 0 && !(s == 0 && r == b.skip_release_item)) st_release(fl + local, (int)(s + 1));
    }
}

// Waveform record of the final level of every instance (block row y = instance).
template <class P>
__global__ void batched_extract_kernel(BatchDev b) {
    const int k = blockIdx.y;
    const InstDev& d = b.inst[k];
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.nth) return;
    const int64_t n = *b.n_steps;
    const int bin = (int)((b.base_bin[k] + n) & 1);
    const int64_t step = b.base_step[k] + n;
    const Planes<P> in = Planes<P>::of(d, bin);
    size_t o = (size_t)j * d.pitch + d.i_e;
    double2 a = in.load(o).phi64(), c = in.load(o + 1).phi64();
    double f = d.f_e;
    double2 w = make_double2((1.0 - f) * a.x + f * c.x, (1.0 - f) * a.y + f * c.y);
    d.wave[(size_t)(step % d.wave_cap) * d.nth + j] = w;
    if (!isfinite(w.x) || !isfinite(w.y)) atomicOr(d.status, (unsigned)ST_NONFINITE);
}

int batched_grid(int prec) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (prec == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_step_kernel<P64>, 128, 0);
    else if (prec == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_step_kernel<P32>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_step_kernel<PK>, 128, 0);
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

void launch_batched_step(cudaStream_t st, int prec, const BatchDev& b, int grid) {
    if (prec == 0) batched_step_kernel<P64><<<grid, 128, 0, st>>>(b);
    else if (prec == 1) batched_step_kernel<P32><<<grid, 128, 0, st>>>(b);
    else batched_step_kernel<PK><<<grid, 128, 0, st>>>(b);
}

void launch_batched_extract(cudaStream_t st, int prec, const BatchDev& b, int max_nth) {
    dim3 g((max_nth + 127) / 128, b.n_inst);
    if (prec == 0) batched_extract_kernel<P64><<<g, 128, 0, st>>>(b);
    else if (prec == 1) batched_extract_kernel<P32><<<g, 128, 0, st>>>(b);
    else batched_extract_kernel<PK><<<g, 128, 0, st>>>(b);
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
