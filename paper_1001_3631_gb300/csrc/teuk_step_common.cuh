// teuk_step_common.cuh -- device building blocks of the Lax-Wendroff step kernels:
// precision policies, node loads/stores, the compensated update, the predictor
// (Eq. 13) and corrector (Eq. 14) bodies.  See teuk_step.cu for the scheme.
#pragma once
#include "teuk_internal.cuh"

namespace teuk {

constexpr int kMaxRows = 1024;   // a block holds one theta column of up to 1024 rows

// ---------------------------------------------------------------- complex
template <typename T>
struct Cx {
    T re, im;
    __device__ __forceinline__ static Cx zero() { return {T(0), T(0)}; }
    __device__ __forceinline__ static Cx half_sum(Cx a, Cx b) {
        return {T(0.5) * (a.re + b.re), T(0.5) * (a.im + b.im)};
    }
};
template <typename T>
__device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return {s * a.re, s * a.im}; }
// Fused multiply-add in the type itself (a plain fma() call on floats would resolve to
// the double overload and run on the FP64 pipe).
__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// acc + (cr + i ci) * z
template <typename T>
__device__ __forceinline__ Cx<T> cmac(Cx<T> acc, T cr, T ci, Cx<T> z) {
    return {tfma(cr, z.re, tfma(-ci, z.im, acc.re)), tfma(cr, z.im, tfma(ci, z.re, acc.im))};
}
// acc + s * z (s real)
template <typename T>
__device__ __forceinline__ Cx<T> rmac(Cx<T> acc, T s, Cx<T> z) {
    return {tfma(s, z.re, acc.re), tfma(s, z.im, acc.im)};
}
// -a
template <typename T>
__device__ __forceinline__ Cx<T> neg(Cx<T> a) { return {-a.re, -a.im}; }

// FP32 complex values in paired instructions (sm_100 and later: FADD2 / FMUL2 / FFMA2
// act on both components of a register pair).  Each component rounds exactly as the
// scalar round-to-nearest operation, so these overloads change no result, only the
// instruction count.
__device__ __forceinline__ float2 pk(Cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ Cx<float> up(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ Cx<float> operator+(Cx<float> a, Cx<float> b) {
    return up(__fadd2_rn(pk(a), pk(b)));
}
// a - b as b * (-1) + a: the product is exact, so this rounds as the subtraction
__device__ __forceinline__ Cx<float> operator-(Cx<float> a, Cx<float> b) {
    return up(__ffma2_rn(bc(-1.0f), pk(b), pk(a)));
}
__device__ __forceinline__ Cx<float> neg(Cx<float> a) { return up(__fmul2_rn(bc(-1.0f), pk(a))); }
__device__ __forceinline__ Cx<float> operator*(float s, Cx<float> a) {
    return up(__fmul2_rn(bc(s), pk(a)));
}
template <>
__device__ __forceinline__ Cx<float> Cx<float>::half_sum(Cx<float> a, Cx<float> b) {
    return up(__fmul2_rn(bc(0.5f), __fadd2_rn(pk(a), pk(b))));
}
// (a + b)/2 + c (the halving is exact, so one fused operation rounds the same)
template <typename T>
__device__ __forceinline__ Cx<T> half_sum_add(Cx<T> a, Cx<T> b, Cx<T> c) {
    return Cx<T>::half_sum(a, b) + c;
}
__device__ __forceinline__ Cx<float> half_sum_add(Cx<float> a, Cx<float> b, Cx<float> c) {
    return up(__ffma2_rn(bc(0.5f), __fadd2_rn(pk(a), pk(b)), pk(c)));
}
__device__ __forceinline__ Cx<float> rmac(Cx<float> acc, float s, Cx<float> z) {
    return up(__ffma2_rn(bc(s), pk(z), pk(acc)));
}

// ---------------------------------------------------------------- precisions
// planes: 16-byte planes per state buffer (the layout in teuk_internal.cuh);
// blocks256: resident blocks per SM that the register budget of the step kernel for
// columns of up to 256 rows aims at (two: at three the FP32 paths fit in 80 registers
// but run no faster, being issue-bound)
struct P64 {
    using T = double;
    static constexpr bool kahan = false;
    static constexpr int planes = 2, blocks256 = 2;
};
struct P32 {
    using T = float;
    static constexpr bool kahan = false;
    static constexpr int planes = 1, blocks256 = 2;
};
struct PK {
    using T = float;
    static constexpr bool kahan = true;
    static constexpr int planes = 2, blocks256 = 2;
};

// Compensated add (Kahan 1965) of both components of a complex value: the represented
// value is hi - c.
__device__ __forceinline__ void kahan_add(Cx<float>& hi, Cx<float>& c, Cx<float> delta) {
    const Cx<float> y = delta - c;
    const Cx<float> t = hi + y;
    c = (t - hi) - y;
    hi = t;
}

// State of one node: Phi, Pi (and, compensated, their c parts).
template <class P>
struct NodeV {
    using T = typename P::T;
    Cx<T> F, Pp;      // hi parts (or the value)
    Cx<T> Fc, Pc;     // compensations (Kahan only; zero otherwise)
    __device__ __forceinline__ static NodeV zero() {
        NodeV n;
        n.F = n.Pp = n.Fc = n.Pc = Cx<T>::zero();
        return n;
    }
    // Phi(this) - Phi(o), accurate for compensated pairs
    __device__ __forceinline__ Cx<T> dphi(const NodeV& o) const {
        if constexpr (P::kahan) return (F - o.F) - (Fc - o.Fc);
        else return F - o.F;
    }
    // gs Phi(this) - Phi(o) and Phi(this) - gs Phi(o) for gs = +-1 (an exact scaling, so
    // these round exactly as dphi of the scaled node)
    __device__ __forceinline__ Cx<T> dphi_sl(T gs, const NodeV& o) const {
        const Cx<T> a = rmac(neg(o.F), gs, F);
        if constexpr (P::kahan) return a - rmac(neg(o.Fc), gs, Fc);
        else return a;
    }
    __device__ __forceinline__ Cx<T> dphi_sr(T gs, const NodeV& o) const {
        const Cx<T> a = rmac(F, -gs, o.F);
        if constexpr (P::kahan) return a - rmac(Fc, -gs, o.Fc);
        else return a;
    }
    __device__ __forceinline__ Cx<T> dpi(const NodeV& o) const {
        if constexpr (P::kahan) return (Pp - o.Pp) - (Pc - o.Pc);
        else return Pp - o.Pp;
    }
    __device__ __forceinline__ double2 phi64() const {
        if constexpr (P::kahan)
            return make_double2((double)F.re - (double)Fc.re, (double)F.im - (double)Fc.im);
        else return make_double2((double)F.re, (double)F.im);
    }
    __device__ __forceinline__ void update(Cx<T> dF, Cx<T> dP) {
        if constexpr (P::kahan) {
            kahan_add(F, Fc, dF);
            kahan_add(Pp, Pc, dP);
        } else {
            F = F + dF; Pp = Pp + dP;
        }
    }
};

// Views of the planes of one ping-pong buffer.
template <class P> struct Planes;
template <> struct Planes<P64> {
    double2* phi; double2* pi;
    __device__ __forceinline__ static Planes of(const InstDev& d, int b) {
        return {(double2*)d.buf[b][0], (double2*)d.buf[b][1]};
    }
    // planes of one column copied to shared memory, `stride` nodes apart
    __device__ __forceinline__ static Planes at(void* base, unsigned stride) {
        return {(double2*)base, (double2*)base + stride};
    }
    __device__ __forceinline__ NodeV<P64> load(size_t o) const {
        NodeV<P64> n;
        double2 a = phi[o], b = pi[o];
        n.F = {a.x, a.y}; n.Pp = {b.x, b.y};
        n.Fc = n.Pc = Cx<double>::zero();
        return n;
    }
    // Phi alone (the theta neighbours of a node)
    __device__ __forceinline__ NodeV<P64> load_phi(size_t o) const {
        NodeV<P64> n = NodeV<P64>::zero();
        double2 a = phi[o];
        n.F = {a.x, a.y};
        return n;
    }
    __device__ __forceinline__ void store(size_t o, const NodeV<P64>& n) const {
        phi[o] = make_double2(n.F.re, n.F.im);
        pi[o] = make_double2(n.Pp.re, n.Pp.im);
    }
};
template <> struct Planes<P32> {
    float4* u;
    __device__ __forceinline__ static Planes of(const InstDev& d, int b) { return {(float4*)d.buf[b][0]}; }
    __device__ __forceinline__ static Planes at(void* base, unsigned) { return {(float4*)base}; }
    __device__ __forceinline__ NodeV<P32> load(size_t o) const {
        NodeV<P32> n;
        float4 a = u[o];
        n.F = {a.x, a.y}; n.Pp = {a.z, a.w};
        n.Fc = n.Pc = Cx<float>::zero();
        return n;
    }
    __device__ __forceinline__ NodeV<P32> load_phi(size_t o) const {
        NodeV<P32> n = NodeV<P32>::zero();
        float2 a = *(const float2*)(u + o);
        n.F = {a.x, a.y};
        return n;
    }
    __device__ __forceinline__ void store(size_t o, const NodeV<P32>& n) const {
        u[o] = make_float4(n.F.re, n.F.im, n.Pp.re, n.Pp.im);
    }
};
template <> struct Planes<PK> {
    float4* hi; float4* c;
    __device__ __forceinline__ static Planes of(const InstDev& d, int b) {
        return {(float4*)d.buf[b][0], (float4*)d.buf[b][1]};
    }
    __device__ __forceinline__ static Planes at(void* base, unsigned stride) {
        return {(float4*)base, (float4*)base + stride};
    }
    __device__ __forceinline__ NodeV<PK> load(size_t o) const {
        NodeV<PK> n;
        float4 a = hi[o], b = c[o];
        n.F = {a.x, a.y}; n.Pp = {a.z, a.w};
        n.Fc = {b.x, b.y}; n.Pc = {b.z, b.w};
        return n;
    }
    __device__ __forceinline__ NodeV<PK> load_phi(size_t o) const {
        NodeV<PK> n = NodeV<PK>::zero();
        float2 a = *(const float2*)(hi + o), b = *(const float2*)(c + o);
        n.F = {a.x, a.y};
        n.Fc = {b.x, b.y};
        return n;
    }
    __device__ __forceinline__ void store(size_t o, const NodeV<PK>& n) const {
        hi[o] = make_float4(n.F.re, n.F.im, n.Pp.re, n.Pp.im);
        c[o] = make_float4(n.Fc.re, n.Fc.im, n.Pc.re, n.Pc.im);
    }
};

// ---------------------------------------------------------------- half nodes
template <typename T>
struct Half { Cx<T> Fb, Pb, dF, dP; };

// Averages and radial differences across the half node i+1/2 (own = column i,
// nb = column i+1).
template <class P>
__device__ __forceinline__ Half<typename P::T> half_prep(const NodeV<P>& own, const NodeV<P>& nb) {
    using T = typename P::T;
    Half<T> h;
    if constexpr (P::kahan) {
        h.Fb = T(0.5) * ((own.F + nb.F) - (own.Fc + nb.Fc));
        h.Pb = T(0.5) * ((own.Pp + nb.Pp) - (own.Pc + nb.Pc));
    } else {
        h.Fb = T(0.5) * (own.F + nb.F);
        h.Pb = T(0.5) * (own.Pp + nb.Pp);
    }
    h.dF = nb.dphi(own);
    h.dP = nb.dpi(own);
    return h;
}

// Predictor output at one half node, plus the inputs the corrector needs from it.
template <typename T>
struct HalfRec { Cx<T> Fb, Pb, dF, dP, Dp, hF, hP; };

// Corrector inputs of one row, combined from the half nodes R = i+1/2 and L = i-1/2.
template <typename T>
struct CRow {
    Cx<T> Hs;        // (dh_Phi_R + dh_Phi_L)/2
    Cx<T> DpS;       // (Dp_R + Dp_L)/2
    Cx<T> FC, PC;    // u~ = (h_R + h_L)/2 for Phi and Pi
    Cx<T> dFc, dPc;  // h_R - h_L for Phi and Pi
};

template <typename T>
__device__ __forceinline__ CRow<T> combine_lr(const HalfRec<T>& R, const HalfRec<T>& L) {
    CRow<T> c;
    c.Hs = Cx<T>::half_sum(R.hF, L.hF);
    c.DpS = Cx<T>::half_sum(R.Dp, L.Dp);
    c.FC = half_sum_add(R.Fb, L.Fb, c.Hs);
    c.PC = half_sum_add(R.Pb, L.Pb, Cx<T>::half_sum(R.hP, L.hP));
    c.dFc = half_sum_add(R.dF, L.dF, R.hF - L.hF);
    c.dPc = half_sum_add(R.dP, L.dP, R.hP - L.hP);
    return c;
}

// (rows past n_theta read the padding of the tables: in bounds, never used)
template <typename T>
__device__ __forceinline__ void load_coefs(const T* tab, size_t pl, size_t o, T* cf) {
#pragma unroll
    for (int k = 0; k < kNCoef; ++k) cf[k] = __ldg(tab + k * pl + o);
}

// The theta table of one row as broadcast pairs (x, x), held in registers by its thread
// for a whole work item (FP32 paths; empty for FP64, which reads 2D tables).
struct ThPair { float2 sin2, cs, V, thp, thm; };
template <class P>
struct RowTab {
    ThPair t;
    __device__ __forceinline__ void load(const ThTab* tab, int j, bool ok) {
        if constexpr (sizeof(typename P::T) == 4) {
            const ThTab h = ok ? tab[j] : ThTab{};
            t = ThPair{bc(h.sin2), bc(h.cs), bc(h.V), bc(h.thp), bc(h.thm)};
        }
    }
};

// FP32 coefficients of the half node i+1/2 (.x) and of the node i (.y) of one column,
// from the column's radial table and the row's theta table (see RTab2), in paired
// instructions.
__device__ __forceinline__ void form_coefs2(const RTab2& t, const ThPair& h, float2* cf) {
    const float2 sig2 = __ffma2_rn(t.naD, h.sin2, t.R2);
    float2 rs = make_float2(rsqrtf(sig2.x), rsqrtf(sig2.y));
    // one Newton step on 1/sqrt: rs (1.5 - (sig2 / 2) rs^2)
    const float2 hr = __fmul2_rn(__fmul2_rn(bc(-0.5f), sig2), rs);
    rs = __fmul2_rn(rs, __ffma2_rn(hr, rs, bc(1.5f)));
    const float2 iS = __fmul2_rn(rs, rs);                // 1/Sigma^2 within a few ulp
    const float2 g = __fmul2_rn(t.Rd, rs);
    const float2 ctre = __fmul2_rn(t.ctr, iS);
    const float2 ctim = __fmul2_rn(__ffma2_rn(t.ctc, h.cs, t.cti), iS);
    cf[C_G] = g;
    cf[C_E1R] = __fmul2_rn(t.nsdt, ctre);
    cf[C_E1I] = __fmul2_rn(t.nsdt, ctim);
    const float2 pb = __ffma2_rn(__fmul2_rn(t.nbb, h.sin2), iS, t.pr);   // pr - bb sin^2 iS
    cf[C_E2R] = __ffma2_rn(ctre, g, __fmul2_rn(pb, iS));
    cf[C_E2I] = __ffma2_rn(ctim, g, __fmul2_rn(t.pi, iS));
    const float2 ws = __fmul2_rn(t.Ds, iS);
    cf[C_EP] = __fmul2_rn(ws, h.thp);
    cf[C_EM] = __fmul2_rn(ws, h.thm);
    cf[C_E3R] = __fmul2_rn(__ffma2_rn(t.nDs, h.V, t.qr), iS);
    cf[C_E3I] = __fmul2_rn(t.qi, iS);
}

// FP64 coefficients of the predictor (half = true, node i+1/2) or the corrector (node i)
// at row j, from the 2D tables.
__device__ __forceinline__ void coefs64(const InstDev& d, bool half, int i, int j, double* cf) {
    load_coefs((const double*)(half ? d.coef_h : d.coef_i), plane_elems(d), node_index(d, i, j), cf);
}

// Eq. (13) at the own half node, as an increment on the averaged state.
template <typename T>
__device__ __forceinline__ HalfRec<T> predictor(const Half<T>& h, Cx<T> Dp, Cx<T> Dm, const T* cf,
                                                T hdt, Cx<T> src) {
    HalfRec<T> r;
    r.Fb = h.Fb; r.Pb = h.Pb; r.dF = h.dF; r.dP = h.dP; r.Dp = Dp;
    r.hF = rmac(rmac(Cx<T>::zero(), -cf[C_G], h.dF), hdt, h.Pb);
    Cx<T> a = rmac(src, cf[C_G], h.dP);
    a = cmac(a, cf[C_E1R], cf[C_E1I], h.Pb);
    a = cmac(a, cf[C_E2R], cf[C_E2I], h.dF);
    a = rmac(a, cf[C_EP], Dp);
    a = rmac(a, -cf[C_EM], Dm);
    a = cmac(a, cf[C_E3R], cf[C_E3I], h.Fb);
    r.hP = a;
    return r;
}

// ---------------------------------------------------------------- source
// dt_sub A_n e^{-i (omega t + phase0)} at t = t_n + off * dt: the predictor's factor
// (off = 0, dt_sub = dt/2) or the corrector's (off = 1/2, dt_sub = dt)
__device__ __forceinline__ double2 source_factor(const InstDev& d, int64_t step, double off,
                                                 double dt_sub) {
    double A = (d.src.amps != nullptr && step < d.src.n_amps) ? d.src.amps[step] : 1.0;
    double t = (double)step * d.dt;
    double sn, cs;
    sincos(d.src.omega * (t + off * d.dt) + d.src.phase0, &sn, &cs);
    double h = dt_sub * A;
    return make_double2(h * cs, -h * sn);
}

// tau at a window node: factor (A e^{-i(omega t + phase0)} and the sub-step's share of
// dt) times the profile, from the column-major copy in the arithmetic type
template <typename T> struct V2T;
template <> struct V2T<float> { using V = float2; };
template <> struct V2T<double> { using V = double2; };

template <typename T>
__device__ __forceinline__ Cx<T> source_at(const void* q, int stride, Cx<T> fac, int a, int b) {
    const typename V2T<T>::V p = ((const typename V2T<T>::V*)q)[(size_t)a * stride + b];
    return {fac.re * p.x - fac.im * p.y, fac.re * p.y + fac.im * p.x};
}

template <typename T>
__device__ __forceinline__ Cx<T> source_half(const SourceDev& s, Cx<T> fac, int i, int j) {
    int a = i - s.h_lo, b = j - s.j_lo;
    if ((unsigned)a < (unsigned)s.nh && (unsigned)b < (unsigned)s.nj)
        return source_at<T>(s.Q_half, s.q_stride, fac, a, b);
    return Cx<T>::zero();
}

template <typename T>
__device__ __forceinline__ Cx<T> source_int(const SourceDev& s, Cx<T> fac, int i, int j) {
    int a = i - s.i_lo, b = j - s.j_lo;
    if ((unsigned)a < (unsigned)s.ni && (unsigned)b < (unsigned)s.nj)
        return source_at<T>(s.Q_int, s.q_stride, fac, a, b);
    return Cx<T>::zero();
}

}  // namespace teuk
