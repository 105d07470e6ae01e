// teuk_step.cu -- the Lax-Wendroff step (Eqs. 13-14) as one fused kernel per step.
//
// Work decomposition: a thread block holds one whole theta column (thread j = row j,
// blockDim = n_theta rounded up to a warp) and streams along r* over a strip of
// columns [c0, c1).  The columns of u^n arrive in a ring of shared-memory slots, filled
// by bulk-async (TMA) copies several columns ahead of use; at each column the block
// computes the predictor (Eq. 13) at the half node just behind it and the corrector
// (Eq. 14) at the column behind that, and stores u^{n+1}.  Radial neighbours are the
// registers of the previous column; the theta neighbours of the input state are read
// from the ring slot, and those of the predictor's results through a small shared
// exchange buffer (one barrier per column).  A strip reads two extra columns, so every
// input is read from HBM about once per step.  The angular ghost
// rows of the pole condition (Sec. 2.2) mirror row 0 / row n_theta-1 with sign +1
// (even |m + s|) or -1 (odd |m + s|): on the averaged state in the predictor, on the half-node
// results in the corrector.
//
// Arithmetic, in differences so that the compensated FP32 state keeps its accuracy (a
// difference of two (hi, c) pairs is formed as (hi_a - hi_b) - (c_a - c_b) before
// anything cancels):
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
// approximated.  The FP32 paths write the angular part ep D+ - em D- in the split form
// A (D+ - D-) + B (D+ + D-) (A = (ep + em)/2, B = (ep - em)/2, see split_angular), with
// the second and two-cell differences formed directly from the state.
#include <type_traits>

#include "teuk_internal.cuh"
#include "teuk_step_common.cuh"

namespace teuk {

// ---------------------------------------------------------------- column ring
// PTX wrappers: mbarrier and the bulk-async copy global -> shared (TMA, untiled form).
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              uint64_t* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(b))
        : "memory");
}
// Bulk prefetch of a global range into L2 (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Orders this thread's view of global memory (generic proxy) before its later bulk copies.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Programmatic dependent launch: wait for the previous grid in the stream (complete and
// its memory visible; a no-op for launches without the attribute), and allow the next
// grid to launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kRingWaitNs = 1000000000ull;  // a slot wait gives up after 1 s

// Columns of the input level (every plane, plus on the FP32 paths the column's radial
// table) are copied into R shared-memory slots by one thread, R - 2 columns
// ahead of use; each slot has an mbarrier that its copy completes.  A column is read
// (own node and theta neighbours) when it arrives and its radial tables one column
// later, so its slot is refilled after the barrier two columns on, when every thread
// has finished with it.  Copies start on 16-byte boundaries with sizes in multiples of
// 16 bytes: a column is n_theta 16-byte nodes at a 512-byte aligned offset, a radial
// table 128 bytes.
template <class P, int R>
struct ColumnRing {
    static constexpr int kSlots = R;
    static constexpr bool kTabs = uses_1d_tables<P>();
    __host__ __device__ static unsigned slot_bytes(int threads) {
        return (unsigned)P::planes * (unsigned)threads * 16u + (kTabs ? (unsigned)sizeof(RTab2) : 0u);
    }

    unsigned char* base;  // R slots: planes [P::planes][stride] of 16-byte nodes, then RTab2
    uint64_t* mbar;       // [R]
    unsigned stride;      // nodes per plane in a slot (the block size)
    unsigned sbytes;
    unsigned phase;       // bit s: parity of the next completion awaited on slot s
    bool late;            // a wait gave up

    __device__ __forceinline__ ColumnRing(unsigned char* b, uint64_t* m)
        : base(b), mbar(m), stride(blockDim.x), sbytes(slot_bytes(blockDim.x)), phase(0), late(false) {}

    // One thread, once per block, before any fill; the block synchronizes afterwards.
    __device__ __forceinline__ void init() const {
        for (int k = 0; k < R; ++k) mbar_init(mbar + k);
        mbar_init_fence();
    }
    __device__ __forceinline__ unsigned char* slot(int s) const { return base + (size_t)s * sbytes; }
    __device__ __forceinline__ Planes<P> planes(int s) const { return Planes<P>::at(slot(s), stride); }
    // One thread: copy column col of buffer bin (and its radial tables) into slot s, and
    // prefetch the column's slices of the source profile into L2 (read once per step,
    // they would otherwise come from DRAM, evicted by the state streaming through L2).
    __device__ __forceinline__ void fill(const InstDev& d, int bin, int col, int s) const {
        if (col == d.fault_col) return;   // testing aid: the slot's phase never completes
        if (!TK_IN(d.status, col, d.nr)) return;   // (checked builds; the waiters time out)
        if (d.src.on) {
            const SourceDev& w = d.src;
            const unsigned cb = (unsigned)w.q_stride * (unsigned)sizeof(typename V2T<typename P::T>::V);
            const int a = col - w.i_lo, h = col - w.h_lo;
            if ((unsigned)a < (unsigned)w.ni) bulk_prefetch_l2((const char*)w.Q_int + (size_t)a * cb, cb);
            if ((unsigned)h < (unsigned)w.nh) bulk_prefetch_l2((const char*)w.Q_half + (size_t)h * cb, cb);
        }
        unsigned char* dst = slot(s);
        const unsigned nb = (unsigned)d.nth * 16u;
        mbar_expect_tx(mbar + s, P::planes * nb + (kTabs ? (unsigned)sizeof(RTab2) : 0u));
        const size_t off = (size_t)col * (size_t)d.pitch * 16u;
#pragma unroll
        for (int q = 0; q < P::planes; ++q)
            bulk_copy_g2s(dst + q * stride * 16u, (const unsigned char*)d.buf[bin][q] + off, nb, mbar + s);
        if constexpr (kTabs) {
            bulk_copy_g2s(dst + P::planes * stride * 16u, d.rtab + col, sizeof(RTab2), mbar + s);
        }
    }
    // Wait for the next copy into slot s.  Once a wait has given up, the thread waits
    // no more (its results are void and the status word says so).
    __device__ __forceinline__ void wait(int s) {
        const unsigned par = (phase >> s) & 1u;
        phase ^= 1u << s;
        if (mbar_try_wait(mbar + s, par) || late) return;
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(mbar + s, par))
            if (global_ns() - t0 > kRingWaitNs) { late = true; return; }
    }
    // Radial table of the column in slot s (FP32 paths).
    __device__ __forceinline__ RTab2 tab2(int s) const {
        RTab2 t{};
        if constexpr (kTabs) {
            const float4* q = (const float4*)(slot(s) + P::planes * stride * 16u);
            float4 v[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) v[k] = q[k];
            t.R2 = {v[0].x, v[0].y};   t.naD = {v[0].z, v[0].w};
            t.Rd = {v[1].x, v[1].y};   t.ctr = {v[1].z, v[1].w};
            t.cti = {v[2].x, v[2].y};  t.ctc = {v[2].z, v[2].w};
            t.pr = {v[3].x, v[3].y};   t.pi = {v[3].z, v[3].w};
            t.nbb = {v[4].x, v[4].y};  t.Ds = {v[4].z, v[4].w};
            t.nDs = {v[5].x, v[5].y};  t.qr = {v[5].z, v[5].w};
            t.qi = {v[6].x, v[6].y};   t.nsdt = {v[6].z, v[6].w};
        }
        return t;
    }
    // After a wait gave up: give every copy still in flight (bounded) time to land, so
    // the block never exits with a copy into its shared memory outstanding.
    __device__ void drain() const {
        const unsigned long long t0 = global_ns();
        for (int k = 0; k < R; ++k)
            while (!mbar_try_wait(mbar + k, ((phase >> k) & 1u) ^ 1u))
                if (global_ns() - t0 > kRingWaitNs) return;
    }
};

// Shared memory of a step block: the ring, then the exchange buffer of the predictor's
// results, [2 (column parity)][threads + 2][4] values (row j at entry j + 1; entries 0
// and n_theta + 1 hold the ghost rows of the pole rule).
template <class P, int R>
struct StepShared {
    using T = typename P::T;
    __host__ __device__ static unsigned xbuf_elems(int threads) { return 2u * ((unsigned)threads + 2u) * 4u; }
    __host__ __device__ static unsigned bytes(int threads) {
        return R * ColumnRing<P, R>::slot_bytes(threads) + xbuf_elems(threads) * (unsigned)sizeof(T);
    }
    __device__ __forceinline__ static T* xbuf(unsigned char* base) {
        return (T*)(base + R * ColumnRing<P, R>::slot_bytes(blockDim.x));
    }
};

// Slots of the ring: six for blocks of up to 512 rows, four for larger blocks (whose
// slots are up to four times bigger than those of 256 rows).
constexpr int kRingS = 6, kRingL = 4;

// One work item: the columns [c0, c1) of one instance for one step, one thread per row.
// Per column c: theta differences of Phi(c), dl = Phi(j+1) - Phi(j) and dlm = Phi(j) -
// Phi(j-1), from the ring slot; predictor at the half node c-1/2; exchange of its
// results with the rows above and below (the one barrier of the column); corrector at
// column c-1.  The first two columns are peeled so the steady-state loop has no
// per-column mode switches, and it is unrolled by two so the rotation of the
// previous / current column is register renaming (by two: measured faster than one,
// three or six on GB300).  Columns c0-1 .. c1 are read.
// kPerStep: the block belongs to a per-step launch (programmatic dependent launch: the
// part before griddepcontrol.wait overlaps the previous step, and the block returns at
// once when a bounded wait of an earlier launch gave up).  Returns false in that case.
// kMov: the kernel serves instances whose particle moves (per-step Gaussian tables);
// the kernels of circular orbits are compiled without that code.
template <class P, int R, bool kPerStep, bool kMov>
__device__ __forceinline__ bool strip_step(const InstDev& d, int64_t step, int bin, int c0,
                                           int c1, ColumnRing<P, R>& ring, typename P::T* xbuf) {
    using T = typename P::T;
    using C = Cx<T>;
    constexpr bool kTabsPath = uses_1d_tables<P>();   // FP32 paths: coefficients from 1D tables
    const int j = threadIdx.x;
    const int nth = d.nth;
    const bool row_ok = j < nth;
    const bool bot = j == 0, top = j == nth - 1;
    // theta neighbours in the slot, the pole rows standing in for the ghost rows: row
    // nth = g * row nth-1 and row -1 = g * row 0 (gp, gm the factors)
    const int jp = j + 1 < nth ? j + 1 : j, jm = j > 0 ? j - 1 : 0;
    const T g = (T)d.ghost;
    const T gp = top ? g : T(1), gm = bot ? g : T(1);
    const T hdt = (T)(0.5 * d.dt), fdt = (T)d.dt;
    const Planes<P> out = Planes<P>::of(d, 1 - bin);
    const unsigned xstride = 4u * (blockDim.x + 2u);
    RowTab<P> rt;
    rt.load(d.thtab, j, row_ok);
    const size_t pitch = (size_t)d.pitch;

    // source: this block's columns against the window
    const SourceDev& sw = d.src;
    const bool src_blk = sw.on &&
                         ((c0 - 1 < sw.i_lo + sw.ni && c1 >= sw.i_lo) ||
                          (c0 - 1 < sw.h_lo + sw.nh && c1 >= sw.h_lo));
    // the step's two source factors, computed once in FP64 (sincos) by two warps, one
    // factor each, and shared already rounded to the arithmetic type
    __shared__ T sfac[4];
    __shared__ int skip;
    if (src_blk) {
        const int w1 = blockDim.x > 32 ? 32 : 0;
        if (threadIdx.x == 0) {
            const double2 f = source_factor<kMov>(d, step, 0.0, 0.5 * d.dt);
            sfac[0] = (T)f.x;
            sfac[1] = (T)f.y;
        }
        if (threadIdx.x == w1) {
            const double2 f = source_factor<kMov>(d, step, 0.5, d.dt);
            sfac[2] = (T)f.x;
            sfac[3] = (T)f.y;
        }
    }
    // Everything above reads only constant data; the state of the previous step (read
    // by the ring, overwritten by this step's stores) is touched only below.
    if constexpr (kPerStep) griddep_wait();
    if (threadIdx.x == 0) {
        // a bounded wait of an earlier launch gave up: the state is void until it is reset
        skip = kPerStep ? (*(volatile unsigned*)d.status & ST_TIMEOUT) != 0 : 0;
        if (!skip) {
            fence_proxy_async_global();
            for (int k = 0; k < c1 - c0 + 2 && k < R; ++k) ring.fill(d, bin, c0 - 1 + k, k);
        }
    }
    __syncthreads();
    if (kPerStep && skip) return false;
    C sp_fac = C::zero(), sc_fac = C::zero();
    if (src_blk) {
        sp_fac = {sfac[0], sfac[1]};
        sc_fac = {sfac[2], sfac[3]};
    }
    // moving particle: this row's angular factors join the step's factors; gr points at
    // the step's radial factors (half nodes, then integer nodes)
    const T* gr = nullptr;
    if constexpr (kMov) {
        if (src_blk && sw.moving && step < sw.n_traj) {
            const int b = j - sw.j_lo;
            T gh = T(0), gi = T(0);
            if ((unsigned)b < (unsigned)sw.nj) {
                const T* gt = (const T*)sw.gt + (size_t)step * 2 * sw.nj + b;
                gh = gt[0];
                gi = gt[sw.nj];
            }
            sp_fac = gh * sp_fac;
            sc_fac = gi * sc_fac;
            gr = (const T*)sw.gr + (size_t)step * (sw.nh + sw.ni);
        }
    }
    const bool ex_blk = c0 - 1 <= d.i_e && d.i_e <= c1 - 1;

    // radial boundary condition: Phi = Pi = 0 at i = 0 and i = nr - 1
    if (row_ok && c0 == 1) out.store(node_index(d, 0, j), NodeV<P>::zero());
    if (row_ok && c1 == d.nr - 1) out.store(node_index(d, d.nr - 1, j), NodeV<P>::zero());

    // own node of the column in slot s (rows past nth read slot padding: their results
    // are never stored or exchanged)
    auto node = [&](int s) { return ring.planes(s).load((size_t)j); };
    // theta differences of Phi in the column in slot s (own node u): forward and backward
    // (expanded angular form) or second and two-cell (split form, see split_angular)
    constexpr bool kSplit = split_angular<P>();
    auto theta_diffs = [&](int s, const NodeV<P>& u, C& dl, C& dlm) {
        const Planes<P> pl = ring.planes(s);
        const NodeV<P> dn = pl.load_phi((size_t)jp), upn = pl.load_phi((size_t)jm);
        if constexpr (kSplit) {
            u.theta_split(gp, dn, gm, upn, dl, dlm);
        } else {
            dl = dn.dphi_sl(gp, u);
            dlm = u.dphi_sr(gm, upn);
        }
    };
    // predictor at the half node h between columns h (ul) and h+1 (ur)
    auto predict = [&](const NodeV<P>& ul, const NodeV<P>& ur, C dll, C dlr, C dlml, C dlmr,
                       const T* cf, C src) {
        const Half<T> hp = half_prep<P>(ul, ur);
        const C Dp = C::half_sum(dll, dlr);     // Fb(j+1) - Fb(j)    (split: Fb(j+1) - 2 Fb(j) + Fb(j-1))
        const C Dm = C::half_sum(dlml, dlmr);   // Fb(j) - Fb(j-1)    (split: Fb(j+1) - Fb(j-1))
        return predictor<T, kSplit>(hp, Dp, Dm, cf, hdt, src);
    };
    // coefficients of column col: the half node col+1/2 into cfh and, on the FP32 paths
    // (formed together in paired instructions), the node col into cfi
    auto coefs = [&](int slot, int col, T* cfh, T* cfi) {
        if constexpr (kTabsPath) {
            float2 cf2[kNCoef];
            form_coefs2(ring.tab2(slot), rt.t, cf2);
#pragma unroll
            for (int k = 0; k < kNCoef; ++k) {
                cfh[k] = cf2[k].x;
                cfi[k] = cf2[k].y;
            }
        } else if constexpr (P::kind == kDF) {
            if (TK_IN(d.status, col, d.nr)) coefs_df(d, true, col, j, (DF*)cfh);
        } else {
            if (TK_IN(d.status, col, d.nr)) coefs64(d, true, col, j, (double*)cfh);
        }
    };
    // corrector at column cc from the half nodes L = cc-1/2 and R = cc+1/2; xb is the
    // exchange buffer of this column's parity, srcc the source term at (cc, j); cfi the
    // node's coefficients on the FP32 paths (the FP64 path reads them here)
    auto correct = [&](const HalfRec<T>& Rh, const HalfRec<T>& Lh, const NodeV<P>& uc,
                       const T* cfi, int cc, T* xb, size_t o, C srcc) {
        const CRow<T> row = combine_lr<T, kSplit>(Rh, Lh);
        // publish this row's exchange entry (the split form needs Hs alone: its averaged
        // differences are the row's own), then read the rows above and below
        T* mine = xb + 4 * (j + 1);
        xpublish<P, kSplit>(xb, mine, row, Rh, Lh, g, row_ok, top, bot);
        __syncthreads();
        C Hs_p, Hs_m, DpS_m;
        xread<P, kSplit>(mine, Hs_p, Hs_m, DpS_m);
        T cf[kNCoef];
        if constexpr (kTabsPath) {
#pragma unroll
            for (int k = 0; k < kNCoef; ++k) cf[k] = cfi[k];
        } else if constexpr (P::kind == kDF) {
            if (TK_IN(d.status, cc, d.nr)) coefs_df(d, false, cc, j, (DF*)cf);
        } else {
            if (TK_IN(d.status, cc, d.nr)) coefs64(d, false, cc, j, (double*)cf);
        }
        C dPhi, dPi;
        corrector_incr<P, kSplit>(row, Hs_p, Hs_m, DpS_m, cf, fdt, srcc, dPhi, dPi);
        if (row_ok && TK_IN(d.status, o, plane_elems(d))) {
            NodeV<P> u = uc;
            u.update(dPhi, dPi);
            out.store(o, u);
        }
    };
    // waveform record of the input level between columns i_e (ul) and i_e + 1 (ur)
    auto extract = [&](const NodeV<P>& ul, const NodeV<P>& ur) {
        if (!row_ok) return;
        double2 a = ul.phi64(), b = ur.phi64();
        double f = d.f_e;
        double2 w = wave_lerp(a, b, f);
        const size_t wi = (size_t)(step % d.wave_cap) * nth + j;
        if (TK_IN(d.status, wi, d.wave_cap * nth)) d.wave[wi] = w;
        if (!isfinite(w.x) || !isfinite(w.y)) atomicOr(d.status, (unsigned)ST_NONFINITE);
    };

    // prologue: columns c0-1 (slot 0) and c0 (slot 1)
    C dl_prev, dlm_prev, dl, dlm;
    ring.wait(0);
    NodeV<P> u_prev = node(0);
    theta_diffs(0, u_prev, dl_prev, dlm_prev);
    ring.wait(1);
    NodeV<P> u_cur = node(1);
    theta_diffs(1, u_cur, dl, dlm);
    // source terms at the half node h and the node i (source blocks only)
    auto src_h = [&](int h) { return source_half<T>(sw, sp_fac, h, j); };
    auto src_i = [&](int i) { return source_int<T>(sw, sc_fac, i, j); };
    // the same for a moving particle: the column's radial factor joins the step's factor
    auto msrc_h = [&](int h) {
        const int a = h - sw.h_lo;
        const T g = (unsigned)a < (unsigned)sw.nh ? gr[a] : T(0);
        return source_half<T>(sw, g * sp_fac, h, j);
    };
    auto msrc_i = [&](int i) {
        const int a = i - sw.i_lo;
        const T g = (unsigned)a < (unsigned)sw.ni ? gr[sw.nh + a] : T(0);
        return source_int<T>(sw, g * sc_fac, i, j);
    };
    T cfh[kNCoef], cfi[kNCoef];
    coefs(0, c0 - 1, cfh, cfi);
    C s_first = C::zero();
    if constexpr (kMov) {
        if (gr) s_first = msrc_h(c0 - 1);
        else if (src_blk) s_first = src_h(c0 - 1);
    } else {
        if (src_blk) s_first = src_h(c0 - 1);
    }
    HalfRec<T> L = predict(u_prev, u_cur, dl_prev, dl, dlm_prev, dlm, cfh, s_first);
    if (ex_blk && d.i_e == c0 - 1) extract(u_prev, u_cur);
    u_prev = u_cur;
    dl_prev = dl;
    dlm_prev = dlm;
    size_t o = node_index(d, c0, j);               // output offset of the corrector's column

    // steady state: column c arrives, predictor at c-1/2, corrector at c-1; the slots
    // hold columns c-2 (sf, free once the column's barrier is passed), c-1 (sp) and c (sc).
    // Three instances of the loop: blocks without source nodes carry no source code; the
    // source blocks (circular orbit: kSrc = 1, moving particle: 2) load the next
    // column's source terms one column ahead.
    auto steady = [&](auto src_kind) {
        constexpr int kSrc = decltype(src_kind)::value;
        auto load_src = [&](int c, C& h, C& i) {
            if constexpr (kSrc == 1) {
                h = src_h(c);
                i = src_i(c);
            } else if constexpr (kSrc == 2 && kMov) {
                h = msrc_h(c);
                i = msrc_i(c);
            }
        };
        C nxt_h = C::zero(), nxt_i = C::zero();
        load_src(c0, nxt_h, nxt_i);
        int sf = 0, sp = 1, sc = 2;
#pragma unroll 2
        for (int c = c0 + 1; c <= c1; ++c) {
            const C s_h = nxt_h, s_i = nxt_i;
            if constexpr (kSrc != 0) {
                if (c < c1) load_src(c, nxt_h, nxt_i);
            }
            ring.wait(sc);
            u_cur = node(sc);
            theta_diffs(sc, u_cur, dl, dlm);
            coefs(sp, c - 1, cfh, cfi);
            const HalfRec<T> Rh = predict(u_prev, u_cur, dl_prev, dl, dlm_prev, dlm, cfh, s_h);
            correct(Rh, L, u_prev, cfi, c - 1, xbuf + (c & 1) * xstride, o, s_i);
            if (threadIdx.x == 0 && c - 2 + R <= c1) ring.fill(d, bin, c - 2 + R, sf);
            if (ex_blk && d.i_e == c - 1) extract(u_prev, u_cur);
            L = Rh;
            u_prev = u_cur;
            dl_prev = dl;
            dlm_prev = dlm;
            o += pitch;
            sf = sp;
            sp = sc;
            sc = sc + 1 == R ? 0 : sc + 1;
        }
    };
    if constexpr (kMov) {
        if (gr) steady(std::integral_constant<int, 2>{});
        else if (src_blk) steady(std::integral_constant<int, 1>{});
        else steady(std::integral_constant<int, 0>{});
    } else {
        if (src_blk) steady(std::integral_constant<int, 1>{});
        else steady(std::integral_constant<int, 0>{});
    }
    if (__syncthreads_or(ring.late)) {
        if (threadIdx.x == 0) {
            ring.drain();
            atomicOr(d.status, (unsigned)ST_TIMEOUT);
        }
        __syncthreads();
        ring.late = false;
    }
    return true;
}

// Three register budgets: columns of up to 256 rows (the common case, P::blocks256
// blocks per SM), of up to 512 rows (one block per SM, 128 registers a thread) and of up
// to 1024 rows.  Dynamic shared memory:
// StepShared<P, R>::bytes(blockDim.x).
// part (may be null): the block's columns are [part[b], part[b+1]) instead of the uniform
// strips; it is written by the host before the launch sequence and never changes while
// a step runs, so it is read before griddepcontrol.wait.
template <class P, int R, bool kMov>
__device__ __forceinline__ void step_body(const InstDev& d, int64_t step, int bin, int strip,
                                          const int* part) {
    extern __shared__ __align__(128) unsigned char step_smem[];
    __shared__ uint64_t mbar[R];
    // the next step's launch may begin now: its blocks become resident as ours retire and
    // run their set-up while this step drains
    griddep_launch_dependents();
    // replayed from a graph: the step is an offset from a base that the host (before the
    // first replay) or the graph's last node (after each replay) sets; it does not change
    // while the graph's steps run
    if (d.step_base) step += *d.step_base;
    ColumnRing<P, R> ring(step_smem, mbar);
    if (threadIdx.x == 0) ring.init();
    __syncthreads();
    int c0, c1;
    if (part) {
        c0 = part[blockIdx.x];
        c1 = part[blockIdx.x + 1];
    } else {
        c0 = 1 + blockIdx.x * strip;
        c1 = min(d.nr - 1, c0 + strip);
    }
    strip_step<P, R, true, kMov>(d, step, bin, c0, c1, ring, StepShared<P, R>::xbuf(step_smem));
}

template <class P, bool kMov>
__global__ void __launch_bounds__(256, P::blocks256) step_kernel_s(InstDev d, int64_t step, int bin, int strip,
                                                                  const int* part) {
    step_body<P, kRingS, kMov>(d, step, bin, strip, part);
}

template <class P, bool kMov>
__global__ void __launch_bounds__(512, 1) step_kernel_m(InstDev d, int64_t step, int bin, int strip,
                                                       const int* part) {
    step_body<P, kRingS, kMov>(d, step, bin, strip, part);
}

template <class P, bool kMov>
__global__ void __launch_bounds__(1024) step_kernel_l(InstDev d, int64_t step, int bin, int strip,
                                                     const int* part) {
    step_body<P, kRingL, kMov>(d, step, bin, strip, part);
}

__global__ void advance_step_kernel(int64_t* base, int64_t k) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *base += k;
}

void launch_advance_step(cudaStream_t st, int64_t* base, int64_t k) {
    advance_step_kernel<<<1, 32, 0, st>>>(base, k);
}

// Waveform record of the state in buffer bin (time level `step`): one thread per row.
template <class P>
__global__ void extract_kernel(InstDev d, int64_t step, int bin) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.nth) return;
    if (!TK_IN(d.status, d.i_e + 1, d.nr) || !TK_IN(d.status, d.i_e, d.nr)) return;
    const Planes<P> in = Planes<P>::of(d, bin);
    double2 a = in.load(node_index(d, d.i_e, j)).phi64();
    double2 b = in.load(node_index(d, d.i_e + 1, j)).phi64();
    double f = d.f_e;
    double2 w = wave_lerp(a, b, f);
    const size_t wi = (size_t)(step % d.wave_cap) * d.nth + j;
    if (TK_IN(d.status, wi, d.wave_cap * d.nth)) d.wave[wi] = w;
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

// Wait until the strips st-1, st, st+1 of the previous step have completed.  That
// covers what this strip reads (one column on each side) and what it overwrites (the
// buffer its neighbours read).  Threads 0..2 poll one neighbour each with acquire
// loads; a wait gives up after spin_limit polls.  Returns false on give-up or abort.
__device__ bool wait_neighbours(const BatchDev& b, const int* fl, int nstrip, int st, int64_t s,
                                int* flag_smem) {
    const int t = threadIdx.x;
    if (t == 0) *flag_smem = 1;
    __syncthreads();
    if (t < 3) {
        int q = st + t - 1;
        if (q >= 0 && q < nstrip) {
            long long it = 0;
            while (ld_acquire(fl + q) < (int)s) {
                if (++it > b.spin_limit || *(volatile int*)b.abort) {
                    *flag_smem = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
    }
    __syncthreads();
    bool ok = *flag_smem != 0;
    __threadfence();
    __syncthreads();
    return ok;
}

// Persistent kernel of one block-size class: blocks grab (step, instance, strip) items
// in step order; an item waits for its radial neighbours of the previous step.  Items
// only wait on items grabbed earlier, so the launch cannot deadlock whatever the
// number of resident blocks.  kMov: some instance of the class has a moving particle.
template <class P, int kMaxThreads, int kMinBlocks, int R, bool kMov>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) batched_step_kernel(BatchDev b) {
    extern __shared__ __align__(128) unsigned char step_smem[];
    __shared__ uint64_t mbar[R];
    __shared__ unsigned long long item;
    __shared__ int flag;
    __shared__ InstDev inst_sm;
    static_assert(sizeof(InstDev) % sizeof(int) == 0, "descriptor copied as ints");
    ColumnRing<P, R> ring(step_smem, mbar);
    typename P::T* xbuf = StepShared<P, R>::xbuf(step_smem);
    if (threadIdx.x == 0) ring.init();
    const int64_t nsteps = *b.n_steps;
    const int64_t total = b.items_per_step * nsteps;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(b.counter, 1ull);
        __syncthreads();
        const unsigned long long g = item;
        if ((int64_t)g >= total || *(volatile int*)b.abort) return;
        const int64_t s = (int64_t)g / b.items_per_step, r = (int64_t)g % b.items_per_step;
        int lo = 0, hi = b.n_inst - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (b.item_base[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const int k = lo;
        const int st = (int)(r - b.item_base[k]);
        if (!TK_IN(b.status, k, b.n_inst) || !TK_IN(b.status, r, b.items_per_step)) return;
        // the item's instance descriptor in shared memory: its fields are then cheap
        // shared loads instead of global loads held in registers (the previous item's
        // readers are past the barrier that ends strip_step)
        for (int q = threadIdx.x; q < (int)(sizeof(InstDev) / sizeof(int)); q += blockDim.x)
            ((int*)&inst_sm)[q] = ((const int*)(b.inst + k))[q];
        __syncthreads();
        const InstDev& d = inst_sm;
        const int strip = b.strip[k], nstrip = b.nstrip[k];
        if (!TK_IN(b.status, st, nstrip)) return;
        int* fl = b.flags + b.item_base[k];
        if (s > 0 && !wait_neighbours(b, fl, nstrip, st, s, &flag)) {
            if (threadIdx.x == 0) {
                atomicOr(b.status, (unsigned)ST_TIMEOUT);
                atomicExch(b.abort, 1);
            }
            return;
        }
        const int c0 = 1 + st * strip;
        const int c1 = min(d.nr - 1, c0 + strip);
        strip_step<P, R, false, kMov>(d, b.base_step[k] + s, (int)((b.base_bin[k] + s) & 1), c0, c1, ring, xbuf);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && !(s == 0 && r == b.skip_release_item))
            st_release(fl + st, (int)(s + 1));
    }
}

// Waveform record of the final level of every instance of the class (block row y).
template <class P>
__global__ void batched_extract_kernel(BatchDev b) {
    const int k = blockIdx.y;
    if (!TK_IN(b.status, k, b.n_inst)) return;
    const InstDev& d = b.inst[k];
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.nth) return;
    if (!TK_IN(d.status, d.i_e + 1, d.nr) || !TK_IN(d.status, d.i_e, d.nr)) return;
    const int64_t n = *b.n_steps;
    const int bin = (int)((b.base_bin[k] + n) & 1);
    const int64_t step = b.base_step[k] + n;
    const Planes<P> in = Planes<P>::of(d, bin);
    double2 a = in.load(node_index(d, d.i_e, j)).phi64();
    double2 c = in.load(node_index(d, d.i_e + 1, j)).phi64();
    double f = d.f_e;
    double2 w = wave_lerp(a, c, f);
    const size_t wi = (size_t)(step % d.wave_cap) * d.nth + j;
    if (TK_IN(d.status, wi, d.wave_cap * d.nth)) d.wave[wi] = w;
    if (!isfinite(w.x) || !isfinite(w.y)) atomicOr(d.status, (unsigned)ST_NONFINITE);
}

template <class P>
static int grid_for(int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the smaller residency of the two variants (with and without moving particles)
    int per2 = 0;
    if (threads <= 256) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_step_kernel<P, 256, P::blocks256, kRingS, false>,
                                                      threads, StepShared<P, kRingS>::bytes(threads));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, batched_step_kernel<P, 256, P::blocks256, kRingS, true>,
                                                      threads, StepShared<P, kRingS>::bytes(threads));
    } else if (threads <= 512) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_step_kernel<P, 512, 1, kRingS, false>,
                                                      threads, StepShared<P, kRingS>::bytes(threads));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, batched_step_kernel<P, 512, 1, kRingS, true>,
                                                      threads, StepShared<P, kRingS>::bytes(threads));
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_step_kernel<P, 1024, 1, kRingL, false>,
                                                      threads, StepShared<P, kRingL>::bytes(threads));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, batched_step_kernel<P, 1024, 1, kRingL, true>,
                                                      threads, StepShared<P, kRingL>::bytes(threads));
    }
    per = per < per2 ? per : per2;
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

int batched_grid(int prec, int threads) {
    if (prec == 0) return grid_for<P64>(threads);
    if (prec == 1) return grid_for<P32>(threads);
    if (prec == 3) return grid_for<PD>(threads);
    return grid_for<PK>(threads);
}

template <class P, bool kMov>
static void launch_batched_m(cudaStream_t st, const BatchDev& b, int grid, int threads) {
    if (threads <= 256)
        batched_step_kernel<P, 256, P::blocks256, kRingS, kMov><<<grid, threads, StepShared<P, kRingS>::bytes(threads), st>>>(b);
    else if (threads <= 512)
        batched_step_kernel<P, 512, 1, kRingS, kMov><<<grid, threads, StepShared<P, kRingS>::bytes(threads), st>>>(b);
    else
        batched_step_kernel<P, 1024, 1, kRingL, kMov><<<grid, threads, StepShared<P, kRingL>::bytes(threads), st>>>(b);
}
template <class P>
static void launch_batched_p(cudaStream_t st, const BatchDev& b, int grid, int threads, bool mov) {
    if (mov) launch_batched_m<P, true>(st, b, grid, threads);
    else launch_batched_m<P, false>(st, b, grid, threads);
}

void launch_batched_step(cudaStream_t st, int prec, const BatchDev& b, int grid, int threads,
                         bool moving) {
    if (prec == 0) launch_batched_p<P64>(st, b, grid, threads, moving);
    else if (prec == 1) launch_batched_p<P32>(st, b, grid, threads, moving);
    else if (prec == 3) launch_batched_p<PD>(st, b, grid, threads, moving);
    else launch_batched_p<PK>(st, b, grid, threads, moving);
}

void launch_batched_extract(cudaStream_t st, int prec, const BatchDev& b, int max_nth) {
    dim3 g((max_nth + 127) / 128, b.n_inst);
    if (prec == 0) batched_extract_kernel<P64><<<g, 128, 0, st>>>(b);
    else if (prec == 1) batched_extract_kernel<P32><<<g, 128, 0, st>>>(b);
    else if (prec == 3) batched_extract_kernel<PD><<<g, 128, 0, st>>>(b);
    else batched_extract_kernel<PK><<<g, 128, 0, st>>>(b);
}

template <class P, bool kMov>
static void launch_step_m(cudaStream_t st, const InstDev& d, int64_t step, int bin, int strip,
                          const int* part) {
    int blocks = (d.nr - 2 + strip - 1) / strip;
    int threads = d.pitch;
    // programmatic dependent launch (see step_body)
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (threads <= 256) {
        cfg.dynamicSmemBytes = StepShared<P, kRingS>::bytes(threads);
        cudaLaunchKernelEx(&cfg, step_kernel_s<P, kMov>, d, step, bin, strip, part);
    } else if (threads <= 512) {
        cfg.dynamicSmemBytes = StepShared<P, kRingS>::bytes(threads);
        cudaLaunchKernelEx(&cfg, step_kernel_m<P, kMov>, d, step, bin, strip, part);
    } else {
        cfg.dynamicSmemBytes = StepShared<P, kRingL>::bytes(threads);
        cudaLaunchKernelEx(&cfg, step_kernel_l<P, kMov>, d, step, bin, strip, part);
    }
}
template <class P>
static void launch_step_p(cudaStream_t st, const InstDev& d, int64_t step, int bin, int strip,
                          const int* part) {
    if (d.src.on && d.src.moving) launch_step_m<P, true>(st, d, step, bin, strip, part);
    else launch_step_m<P, false>(st, d, step, bin, strip, part);
}

template <class P>
static int resident_p(int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (threads <= 256)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel_s<P, false>, threads,
                                                      StepShared<P, kRingS>::bytes(threads));
    else if (threads <= 512)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel_m<P, false>, threads,
                                                      StepShared<P, kRingS>::bytes(threads));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel_l<P, false>, threads,
                                                      StepShared<P, kRingL>::bytes(threads));
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}

int step_resident_blocks(int prec, int threads) {
    if (prec == 0) return resident_p<P64>(threads);
    if (prec == 1) return resident_p<P32>(threads);
    if (prec == 3) return resident_p<PD>(threads);
    return resident_p<PK>(threads);
}

void launch_step(cudaStream_t st, const InstDev& d, int64_t step, int bin, int strip,
                 const int* part) {
    if (d.prec == 0) launch_step_p<P64>(st, d, step, bin, strip, part);
    else if (d.prec == 1) launch_step_p<P32>(st, d, step, bin, strip, part);
    else if (d.prec == 3) launch_step_p<PD>(st, d, step, bin, strip, part);
    else launch_step_p<PK>(st, d, step, bin, strip, part);
}

// Opt the step kernels in to the dynamic shared memory of their largest blocks (on the
// current device; called when a context is created).
template <class P, bool kMov>
static cudaError_t prepare_m() {
    const int s = (int)StepShared<P, kRingS>::bytes(256), m = (int)StepShared<P, kRingS>::bytes(512),
              l = (int)StepShared<P, kRingL>::bytes(1024);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(step_kernel_s<P, kMov>, a, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel_m<P, kMov>, a, m);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel_l<P, kMov>, a, l);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batched_step_kernel<P, 256, P::blocks256, kRingS, kMov>, a, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batched_step_kernel<P, 512, 1, kRingS, kMov>, a, m);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batched_step_kernel<P, 1024, 1, kRingL, kMov>, a, l);
    return e;
}
template <class P>
static cudaError_t prepare_p() {
    cudaError_t e = prepare_m<P, false>();
    if (e == cudaSuccess) e = prepare_m<P, true>();
    return e;
}

cudaError_t prepare_step_kernels() {
    cudaError_t e = prepare_p<P64>();
    if (e == cudaSuccess) e = prepare_p<P32>();
    if (e == cudaSuccess) e = prepare_p<PK>();
    if (e == cudaSuccess) e = prepare_p<PD>();
    return e;
}

void launch_extract(cudaStream_t st, const InstDev& d, int64_t step, int bin) {
    int blocks = (d.nth + 127) / 128;
    if (d.prec == 0) extract_kernel<P64><<<blocks, 128, 0, st>>>(d, step, bin);
    else if (d.prec == 1) extract_kernel<P32><<<blocks, 128, 0, st>>>(d, step, bin);
    else if (d.prec == 3) extract_kernel<PD><<<blocks, 128, 0, st>>>(d, step, bin);
    else extract_kernel<PK><<<blocks, 128, 0, st>>>(d, step, bin);
}

}  // namespace teuk
