// teuk_resident.cu -- the Lax-Wendroff step (Eqs. 13-14) of one instance whose grid is
// small enough to stay in the GPU's shared memory: one cooperative launch advances it
// n steps.
//
// Work decomposition: block b owns the r* columns [c0, c1) for the whole launch and
// holds them, with h halo columns on each side, in shared memory ([c0 - h, c1 + h), local
// index q = col - (c0 - h)).  Thread-column k (threads of one local column, one theta
// row each; a thread serves every KT-th thread-column when the block has fewer threads
// than nodes) computes the predictor (Eq. 13) at the half node between local columns k
// and k+1 and the corrector (Eq. 14) at node k, from the half-node results of k-1 and k,
// which pass through shared memory.  After
// each step the region of valid data shrinks by one column per side, so a block runs h
// steps between exchanges; it then publishes its first and last h owned columns to a
// global exchange buffer, releases its flag, and reads the neighbours' columns into its
// halos once their flags say they are published.  Waits are bounded (1 s of
// %globaltimer): one that gives up sets the status word and an abort flag, and every
// block returns.  The cooperative launch guarantees that all blocks are resident at once
// (the launch is refused otherwise), so no block waits on one that is not running.
//
// The per-node arithmetic is that of the streaming kernel (teuk_step.cu, shared through
// teuk_step_common.cuh) in the same order, so the results equal those of one launch per
// step.  Coefficients are formed (FP32 paths) or read (FP64, double-float) once per
// launch and kept in shared memory; the state is read from HBM once at the start and
// written once at the end.
#include <algorithm>

#include "teuk_internal.cuh"
#include "teuk_step_common.cuh"

namespace teuk {

namespace {

constexpr int kResMaxThreads = 512;
constexpr int kResMaxHalo = 4;             // steps between exchanges, at most
constexpr int kResMaxBps = 4;              // blocks per SM a plan may aim at
constexpr unsigned long long kResWaitNs = 1000000000ull;   // a halo wait gives up after 1 s

__device__ __forceinline__ unsigned long long res_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int res_ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void res_fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// Release store of a flag: the block's earlier stores (ordered before this thread's store
// by the barrier that precedes it) become visible to a reader that acquires the flag.
__device__ __forceinline__ void res_st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Shared-memory layout of a block with ncol local columns, nk = ncol - 1 thread-columns
// and `pitch` rows (all sizes in bytes, each region 16-byte aligned):
//   S   state  [planes][ncol][pitch] 16-byte nodes
//   HR  half-node records [nk][pitch] HalfRec<T>
//   X   corrector exchange [nk][pitch + 2][4] T
//   CF  coefficients [nk][pitch][2 kNCoef] T (half node, then node)
template <class P>
struct ResLayout {
    using T = typename P::T;
    __host__ __device__ static size_t up16(size_t b) { return (b + 15) / 16 * 16; }
    __host__ __device__ static size_t s_bytes(int ncol, int pitch) {
        return (size_t)P::planes * ncol * pitch * 16;
    }
    __host__ __device__ static size_t hr_bytes(int ncol, int pitch) {
        return up16((size_t)(ncol - 1) * pitch * sizeof(HalfRec<T>));
    }
    __host__ __device__ static size_t x_bytes(int ncol, int pitch) {
        return up16((size_t)(ncol - 1) * (pitch + 2) * 4 * sizeof(T));
    }
    __host__ __device__ static size_t cf_bytes(int ncol, int pitch) {
        return up16((size_t)(ncol - 1) * pitch * 2 * kNCoef * sizeof(T));
    }
    __host__ __device__ static size_t bytes(int ncol, int pitch) {
        return s_bytes(ncol, pitch) + hr_bytes(ncol, pitch) + x_bytes(ncol, pitch) + cf_bytes(ncol, pitch);
    }
};

}  // namespace

// Owned columns [c0, c1) of block b: the n_rstar - 2 interior columns split into nb runs
// whose lengths differ by at most one.
__host__ __device__ inline void res_cols(const ResidentArgs& r, int b, int* c0, int* c1) {
    const int cols = r.d.nr - 2;
    const int base = cols / r.nb, extra = cols % r.nb;   // the first `extra` blocks own base + 1
    *c0 = 1 + b * base + (b < extra ? b : extra);
    *c1 = *c0 + base + (b < extra ? 1 : 0);
}

template <class P>
__global__ void __launch_bounds__(kResMaxThreads, 1) resident_kernel(ResidentArgs r) {
    using T = typename P::T;
    using C = Cx<T>;
    constexpr bool kSplit = split_angular<P>();
    constexpr bool kTabsPath = uses_1d_tables<P>();
    extern __shared__ __align__(128) unsigned char res_smem[];
    __shared__ T sfac[2][kResMaxHalo][4];   // [interval parity][step of the interval][4]
    __shared__ int late_any;
    const InstDev& d = r.d;
    const int b = blockIdx.x, h = r.h, pitch = d.pitch, nth = d.nth, nr = d.nr;
    int c0, c1;
    res_cols(r, b, &c0, &c1);
    const int ncol = (c1 - c0) + 2 * h, nk = ncol - 1;
    const int t = threadIdx.x;
    // thread (k0, j): row j of the thread-columns k0, k0 + KT, k0 + 2 KT, ... (< nk)
    const int j = t % pitch, k0 = t / pitch, KT = (int)blockDim.x / pitch;
    const bool row_ok = j < nth;
    const bool bot = j == 0, top = j == nth - 1;
    const int jp = j + 1 < nth ? j + 1 : j, jm = j > 0 ? j - 1 : 0;
    const T g = (T)d.ghost;
    const T gp = top ? g : T(1), gm = bot ? g : T(1);
    const T hdt = (T)(0.5 * d.dt), fdt = (T)d.dt;
    const bool has_l = b > 0, has_r = b < r.nb - 1;

    using L = ResLayout<P>;
    unsigned char* sm = res_smem;
    const Planes<P> S = Planes<P>::at(sm, (unsigned)(ncol * pitch));
    HalfRec<T>* HR = (HalfRec<T>*)(sm + L::s_bytes(ncol, pitch));
    T* X = (T*)(sm + L::s_bytes(ncol, pitch) + L::hr_bytes(ncol, pitch));
    T* CF = (T*)(sm + L::s_bytes(ncol, pitch) + L::hr_bytes(ncol, pitch) + L::x_bytes(ncol, pitch));
    auto sidx = [&](int q, int jj) { return (size_t)q * pitch + jj; };
    // raw 16-byte node copies between global planes (glim nodes a plane) and the shared
    // planes
    auto copy_in = [&](const unsigned char* const* src_planes, size_t src_node, size_t dst_node, bool bypass,
                       size_t glim) {
        if (!TK_IN(d.status, src_node, glim) || !TK_IN(d.status, dst_node, (size_t)ncol * pitch)) return;
#pragma unroll
        for (int p = 0; p < P::planes; ++p) {
            const float4* s = (const float4*)src_planes[p] + src_node;
            float4* dd = (float4*)(sm + (size_t)p * ncol * pitch * 16) + dst_node;
            *dd = bypass ? __ldcg(s) : *s;
        }
    };
    auto copy_out = [&](unsigned char* const* dst_planes, size_t src_node, size_t dst_node, size_t glim) {
        if (!TK_IN(d.status, dst_node, glim) || !TK_IN(d.status, src_node, (size_t)ncol * pitch)) return;
#pragma unroll
        for (int p = 0; p < P::planes; ++p) {
            const float4* s = (const float4*)(sm + (size_t)p * ncol * pitch * 16) + src_node;
            __stcg((float4*)dst_planes[p] + dst_node, *s);
        }
    };

    // ---- start: the coefficients of every thread-column's half node col+1/2 and node col
    // (constant data), then the state of the local columns [0, ncol) that exist, from
    // buffer bin.  A blocked launch releases the next one at once and waits for the
    // previous one (griddepcontrol; no-ops for a launch without programmatic dependence)
    // only before it touches the state.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    RowTab<P> rt;
    rt.load(d.thtab, j, row_ok);
    for (int k = k0; k < nk; k += KT) {
        const int col = c0 - h + k;
        if (col < 0 || col > nr - 1) continue;
        T* mine = CF + sidx(k, j) * 2 * kNCoef;
        if constexpr (kTabsPath) {
            float2 cf2[kNCoef];
            form_coefs2(d.rtab[col], rt.t, cf2);
#pragma unroll
            for (int q = 0; q < kNCoef; ++q) {
                mine[q] = cf2[q].x;
                mine[kNCoef + q] = cf2[q].y;
            }
        } else if constexpr (P::kind == kDF) {
            coefs_df(d, true, col, j, (DF*)mine);
            coefs_df(d, false, col, j, (DF*)(mine + kNCoef));
        } else {
            coefs64(d, true, col, j, (double*)mine);
            coefs64(d, false, col, j, (double*)(mine + kNCoef));
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    {
        const unsigned char* in[2] = {(const unsigned char*)d.buf[r.bin][0],
                                      (const unsigned char*)d.buf[r.bin][P::planes - 1]};
        for (int idx = t; idx < ncol * pitch; idx += blockDim.x) {
            const int q = idx / pitch, jj = idx % pitch, cc = c0 - h + q;
            if (cc >= 0 && cc <= nr - 1) copy_in(in, (size_t)cc * pitch + jj, sidx(q, jj), false, plane_elems(d));
        }
    }
    // source: does this block meet the window (its local columns, halos included)?
    const SourceDev& sw = d.src;
    const int lo = c0 - h, hi = c1 + h;   // local columns [lo, hi)
    const bool src_blk = sw.on && ((lo < sw.i_lo + sw.ni && hi > sw.i_lo) || (lo < sw.h_lo + sw.nh && hi > sw.h_lo));
    const int w1 = blockDim.x > 32 ? 32 : 0;
    // source factors of the hs steps from `step` (an exchange interval), one FP64 factor a
    // thread in the second warp, ahead of the interval (off the steps' critical path)
    auto factors = [&](int64_t step, int hs, int ip) {
        const int q = t - w1;
        if (!src_blk || q < 0 || q >= 2 * hs) return;
        const double2 f = (q & 1) ? source_factor<false>(d, step + q / 2, 0.5, d.dt)
                                  : source_factor<false>(d, step + q / 2, 0.0, 0.5 * d.dt);
        sfac[ip][q / 2][2 * (q & 1)] = (T)f.x;
        sfac[ip][q / 2][2 * (q & 1) + 1] = (T)f.y;
    };
    // extraction: the block holding i_e (block 0 also a record between nodes 0 and 1)
    const bool ex_blk = (b == 0 ? d.i_e < c1 : (c0 <= d.i_e && d.i_e < c1));
    const int qe = d.i_e - (c0 - h);
    auto record = [&](int64_t level) {
        if (!ex_blk || !row_ok || t >= pitch) return;
        const double2 a = S.load(sidx(qe, j)).phi64(), c = S.load(sidx(qe + 1, j)).phi64();
        const double2 w = wave_lerp(a, c, d.f_e);
        const size_t wi = (size_t)(level % d.wave_cap) * nth + j;
        if (TK_IN(d.status, wi, d.wave_cap * nth)) d.wave[wi] = w;
        if (!isfinite(w.x) || !isfinite(w.y)) atomicOr(d.status, (unsigned)ST_NONFINITE);
    };
    // exchange slots: plane p, slot, block, side (0: first h owned, 1: last h owned)
    const size_t xplane = (size_t)2 * r.nb * 2 * h * pitch;   // nodes per plane
    unsigned char* xp[2] = {r.xg, r.xg + (P::planes - 1) * xplane * 16};
    auto xnode = [&](int slot, int blk, int side, int qq, int jj) {
        return (((size_t)slot * r.nb + blk) * 2 + side) * h * pitch + (size_t)qq * pitch + jj;
    };
    // bounded wait until flag[blk] >= v; false if it gave up (or another block did).  The
    // flag is polled with relaxed loads (the abort flag and the clock every 256 polls),
    // and one acquire fence orders the halo reads after the poll that saw it.
    auto wait_flag = [&](int blk, int v) {
        const int* f = r.flags + (size_t)blk * kResFlagStride;
        const unsigned long long t0 = res_ns();
        for (unsigned it = 1;; ++it) {
            if (res_ld_relaxed(f) >= v) break;
            __nanosleep(64);
            if ((it & 63u) == 0 && (*(volatile int*)r.abort || res_ns() - t0 > kResWaitNs)) return false;
        }
        res_fence_acq_rel();
        return true;
    };
    // one thread waits for each neighbour (threads 0 and w1, in different warps)
    auto wait_neighbours = [&](int v) {
        bool late = false;
        if (t == 0 && has_l && !wait_flag(b - 1, v)) late = true;
        if (t == w1 && has_r && !wait_flag(b + 1, v)) late = true;
        if (late) late_any = 1;
        __syncthreads();
        const bool stop = late_any != 0;
        if (stop && t == 0) {
            atomicOr(d.status, (unsigned)ST_TIMEOUT);
            atomicExch(r.abort, 1);
        }
        return !stop;
    };
    if (t == 0) late_any = 0;
    factors(r.step0, (int)(r.n < h ? r.n : h), 0);
    __syncthreads();
    // the initial halos are loaded: neighbours may overwrite the level they read from
    if (t == 0) res_st_release(r.flags + (size_t)b * kResFlagStride, 1);

    int64_t done = 0;
    int exch = 0;
    while (done < r.n) {
        const int hs = (int)((r.n - done) < h ? (r.n - done) : h);
        const int ip = exch & 1;   // factor slot of this interval
        for (int s = 0; s < hs; ++s) {
            const int64_t step = r.step0 + done + s;
            record(step);
            // the predictor works on the half nodes between local columns k and k+1 with
            // k in [s, nk - s); the corrector on the nodes k in [s + 1, nk - s)
            auto pact = [&](int k) {
                const int col = c0 - h + k;
                return k >= s && k < nk - s && col >= 0 && col <= nr - 2;
            };
            auto cact = [&](int k) {
                const int col = c0 - h + k;
                return k >= s + 1 && k < nk - s && col >= 1 && col <= nr - 2;
            };
            // P1: predictor (Eq. 13)
            for (int k = k0; k < nk; k += KT) {
                if (!pact(k)) continue;
                const int col = c0 - h + k;
                const NodeV<P> ul = S.load(sidx(k, j)), ur = S.load(sidx(k + 1, j));
                C dll, dlml, dlr, dlmr;
                {
                    const NodeV<P> dn = S.load_phi(sidx(k, jp)), upn = S.load_phi(sidx(k, jm));
                    if constexpr (kSplit) {
                        ul.theta_split(gp, dn, gm, upn, dll, dlml);
                    } else {
                        dll = dn.dphi_sl(gp, ul);
                        dlml = ul.dphi_sr(gm, upn);
                    }
                }
                {
                    const NodeV<P> dn = S.load_phi(sidx(k + 1, jp)), upn = S.load_phi(sidx(k + 1, jm));
                    if constexpr (kSplit) {
                        ur.theta_split(gp, dn, gm, upn, dlr, dlmr);
                    } else {
                        dlr = dn.dphi_sl(gp, ur);
                        dlmr = ur.dphi_sr(gm, upn);
                    }
                }
                C s_h = C::zero();
                if (src_blk) s_h = source_half<T>(sw, C{sfac[ip][s][0], sfac[ip][s][1]}, col, j);
                T cf[kNCoef];
#pragma unroll
                for (int q = 0; q < kNCoef; ++q) cf[q] = CF[sidx(k, j) * 2 * kNCoef + q];
                const Half<T> hp = half_prep<P>(ul, ur);
                const C Dp = C::half_sum(dll, dlr);
                const C Dm = C::half_sum(dlml, dlmr);
                HR[sidx(k, j)] = predictor<T, kSplit>(hp, Dp, Dm, cf, hdt, s_h);
            }
            __syncthreads();
            // P2: combine the half nodes on both sides of node k, publish the exchange entry
            for (int k = k0; k < nk; k += KT) {
                if (!cact(k)) continue;
                const HalfRec<T> Rh = HR[sidx(k, j)], Lh = HR[sidx(k - 1, j)];
                const CRow<T> row = combine_lr<T, kSplit>(Rh, Lh);
                T* xb = X + (size_t)k * (pitch + 2) * 4;
                xpublish<P, kSplit>(xb, xb + 4 * (j + 1), row, Rh, Lh, g, row_ok, top, bot);
            }
            __syncthreads();
            // P3: corrector (Eq. 14) at node k, in place (this step's state is no longer read)
            for (int k = k0; k < nk; k += KT) {
                const int col = c0 - h + k;
                if (cact(k) && row_ok) {
                    const HalfRec<T> Rh = HR[sidx(k, j)], Lh = HR[sidx(k - 1, j)];
                    const CRow<T> row = combine_lr<T, kSplit>(Rh, Lh);
                    C Hs_p, Hs_m, DpS_m;
                    xread<P, kSplit>(X + (size_t)k * (pitch + 2) * 4 + 4 * (j + 1), Hs_p, Hs_m, DpS_m);
                    C s_i = C::zero();
                    if (src_blk) s_i = source_int<T>(sw, C{sfac[ip][s][2], sfac[ip][s][3]}, col, j);
                    T cf[kNCoef];
#pragma unroll
                    for (int q = 0; q < kNCoef; ++q) cf[q] = CF[sidx(k, j) * 2 * kNCoef + kNCoef + q];
                    C dPhi, dPi;
                    corrector_incr<P, kSplit>(row, Hs_p, Hs_m, DpS_m, cf, fdt, s_i, dPhi, dPi);
                    NodeV<P> u = S.load(sidx(k, j));
                    u.update(dPhi, dPi);
                    S.store(sidx(k, j), u);
                }
                // radial boundary condition: Phi = Pi = 0 at columns 0 and nr - 1
                if (row_ok && k >= s && k < nk - s) {
                    if (col == 0) S.store(sidx(k, j), NodeV<P>::zero());
                    if (col + 1 == nr - 1) S.store(sidx(k + 1, j), NodeV<P>::zero());
                }
            }
            __syncthreads();
        }
        done += hs;
        if (done >= r.n) break;
        // exchange: publish the first and last h owned columns (the barrier, then one release
        // store of the flag), then read the neighbours' columns into the halos once their
        // flags say so
        ++exch;
        const int slot = exch & 1;
        for (int idx = t; idx < 2 * h * pitch; idx += blockDim.x) {
            const int side = idx / (h * pitch), rem = idx % (h * pitch), qq = rem / pitch, jj = rem % pitch;
            const int q = side == 0 ? h + qq : ncol - 2 * h + qq;
            copy_out(xp, sidx(q, jj), xnode(slot, b, side, qq, jj), xplane);
        }
        __syncthreads();
        if (t == 0 && b != r.skip_publish) res_st_release(r.flags + (size_t)b * kResFlagStride, exch + 1);
        // the next interval's source factors, while the neighbours' columns are awaited
        factors(r.step0 + done, (int)((r.n - done) < h ? (r.n - done) : h), exch & 1);
        if (!wait_neighbours(exch + 1)) return;
        for (int idx = t; idx < 2 * h * pitch; idx += blockDim.x) {
            const int side = idx / (h * pitch), rem = idx % (h * pitch), qq = rem / pitch, jj = rem % pitch;
            if (side == 0 ? !has_l : !has_r) continue;
            // the left neighbour's last h owned columns are this block's local 0 .. h-1,
            // the right neighbour's first h are local ncol - h .. ncol - 1
            const int nbk = side == 0 ? b - 1 : b + 1;
            const int q = side == 0 ? qq : ncol - h + qq;
            const unsigned char* src[2] = {xp[0], xp[1]};
            copy_in(src, xnode(slot, nbk, 1 - side, qq, jj), sidx(q, jj), true, xplane);
        }
        __syncthreads();
    }
    // (the record of the final level is taken by the extraction kernel after the launch)
    // ---- end: the owned columns (and the grid's boundary columns at the two ends) into
    // buffer obin, once the neighbours have read their initial halos from buffer bin
    if (!r.no_wait && !wait_neighbours(1)) return;
    unsigned char* out[2] = {(unsigned char*)d.buf[r.obin][0], (unsigned char*)d.buf[r.obin][P::planes - 1]};
    const int qlo = b == 0 ? h - 1 : h, qhi = (b == r.nb - 1) ? ncol - h + 1 : ncol - h;
    for (int idx = t; idx < (qhi - qlo) * pitch; idx += blockDim.x) {
        const int q = qlo + idx / pitch, jj = idx % pitch, cc = c0 - h + q;
        copy_out(out, sidx(q, jj), (size_t)cc * pitch + jj, plane_elems(d));
    }
}

// ---------------------------------------------------------------- host side

template <class P>
static cudaError_t res_occupancy(int threads, size_t smem, int* per_sm) {
    cudaError_t e = cudaFuncSetAttribute(resident_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, resident_kernel<P>, threads, smem);
}

template <class P>
static bool res_plan_p(int nr, int pitch, int h, int bps, ResidentPlan* plan) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int cols = nr - 2;
    const int slots = (sms > 0 ? sms : 1) * bps;
    // the fewest columns per block (from cols / (SMs x bps) up) such that all blocks are
    // resident at once
    for (int W = (cols + slots - 1) / slots; W <= cols; ++W) {
        const int nb = (cols + W - 1) / W;
        if (cols / nb < h) continue;                     // every block owns >= h columns
        const int ncol = W + 2 * h;
        if (pitch > kResMaxThreads) return false;
        const int kt = std::min(kResMaxThreads / pitch, ncol - 1);   // thread-columns
        const int threads = kt * pitch;
        const size_t smem = ResLayout<P>::bytes(ncol, pitch);
        if (smem > 227 * 1024) return false;
        int per = 0;
        if (res_occupancy<P>(threads, smem, &per) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if ((int64_t)per * sms >= nb) {
            plan->nb = nb;
            plan->threads = threads;
            plan->smem = smem;
            plan->h = h;
            plan->bps = bps;
            return true;
        }
    }
    return false;
}

bool resident_plan(int prec, int nr, int pitch, int h, int bps, ResidentPlan* plan) {
    if (h < 1 || h > kResMaxHalo || nr < 4 || bps < 1 || bps > kResMaxBps) return false;
    if (prec == 0) return res_plan_p<P64>(nr, pitch, h, bps, plan);
    if (prec == 1) return res_plan_p<P32>(nr, pitch, h, bps, plan);
    if (prec == 3) return res_plan_p<PD>(nr, pitch, h, bps, plan);
    return res_plan_p<PK>(nr, pitch, h, bps, plan);
}

template <class P>
static cudaError_t launch_res_p(cudaStream_t st, const ResidentArgs& a, const ResidentPlan& plan,
                                bool cooperative) {
    ResidentArgs arg = a;
    if (cooperative) {
        void* params[] = {&arg};
        return cudaLaunchCooperativeKernel((const void*)resident_kernel<P>, dim3(plan.nb), dim3(plan.threads),
                                           params, plan.smem, st);
    }
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.nb);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, resident_kernel<P>, arg);
}

cudaError_t launch_resident(cudaStream_t st, const ResidentArgs& a, const ResidentPlan& plan, bool cooperative) {
    switch (a.d.prec) {
        case 0: return launch_res_p<P64>(st, a, plan, cooperative);
        case 1: return launch_res_p<P32>(st, a, plan, cooperative);
        case 3: return launch_res_p<PD>(st, a, plan, cooperative);
        default: return launch_res_p<PK>(st, a, plan, cooperative);
    }
}

}  // namespace teuk
