// teuk_step_common.cuh -- device building blocks of the Lax-Wendroff step kernels:
// precision policies, node loads/stores, the compensated update, the predictor
// (Eq. 13) and corrector (Eq. 14) bodies.  See teuk_step.cu for the scheme.
#pragma once
#include "teuk_internal.cuh"

namespace teuk {

constexpr unsigned kFull = 0xffffffffu;

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
// acc + (cr + i ci) * z
template <typename T>
__device__ __forceinline__ Cx<T> cmac(Cx<T> acc, T cr, T ci, Cx<T> z) {
    return {fma(cr, z.re, fma(-ci, z.im, acc.re)), fma(cr, z.im, fma(ci, z.re, acc.im))};
}
// acc + s * z (s real)
template <typename T>
__device__ __forceinline__ Cx<T> rmac(Cx<T> acc, T s, Cx<T> z) {
    return {fma(s, z.re, acc.re), fma(s, z.im, acc.im)};
}

__device__ __forceinline__ float shfl_down_t(float v) { return __shfl_down_sync(kFull, v, 1); }
__device__ __forceinline__ double shfl_down_t(double v) { return __shfl_down_sync(kFull, v, 1); }
__device__ __forceinline__ float shfl_up_t(float v) { return __shfl_up_sync(kFull, v, 1); }
__device__ __forceinline__ double shfl_up_t(double v) { return __shfl_up_sync(kFull, v, 1); }
template <typename T>
__device__ __forceinline__ Cx<T> shfl_down_c(Cx<T> a) { return {shfl_down_t(a.re), shfl_down_t(a.im)}; }
template <typename T>
__device__ __forceinline__ Cx<T> shfl_up_c(Cx<T> a) { return {shfl_up_t(a.re), shfl_up_t(a.im)}; }

// ---------------------------------------------------------------- precisions
struct P64 { using T = double; static constexpr bool kahan = false; };
struct P32 { using T = float; static constexpr bool kahan = false; };
struct PK  { using T = float; static constexpr bool kahan = true; };

// Compensated add (Kahan 1965): the represented value is hi - c.
__device__ __forceinline__ void kahan_add(float& hi, float& c, float delta) {
    float y = __fsub_rn(delta, c);
    float t = __fadd_rn(hi, y);
    c = __fsub_rn(__fsub_rn(t, hi), y);
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
    __device__ __forceinline__ void scale(T s) {  // s = +-1: exact
        F = s * F; Pp = s * Pp;
        if constexpr (P::kahan) { Fc = s * Fc; Pc = s * Pc; }
    }
    __device__ __forceinline__ NodeV shfl_down() const {
        NodeV n;
        n.F = shfl_down_c(F); n.Pp = shfl_down_c(Pp);
        if constexpr (P::kahan) { n.Fc = shfl_down_c(Fc); n.Pc = shfl_down_c(Pc); }
        else { n.Fc = n.Pc = Cx<T>::zero(); }
        return n;
    }
    // Phi(this) - Phi(o), accurate for compensated pairs
    __device__ __forceinline__ Cx<T> dphi(const NodeV& o) const {
        if constexpr (P::kahan) return (F - o.F) - (Fc - o.Fc);
        else return F - o.F;
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
            kahan_add(F.re, Fc.re, dF.re); kahan_add(F.im, Fc.im, dF.im);
            kahan_add(Pp.re, Pc.re, dP.re); kahan_add(Pp.im, Pc.im, dP.im);
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
    __device__ __forceinline__ NodeV<P64> load(size_t o) const {
        NodeV<P64> n;
        double2 a = phi[o], b = pi[o];
        n.F = {a.x, a.y}; n.Pp = {b.x, b.y};
        n.Fc = n.Pc = Cx<double>::zero();
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
    __device__ __forceinline__ NodeV<P32> load(size_t o) const {
        NodeV<P32> n;
        float4 a = u[o];
        n.F = {a.x, a.y}; n.Pp = {a.z, a.w};
        n.Fc = n.Pc = Cx<float>::zero();
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
    __device__ __forceinline__ NodeV<PK> load(size_t o) const {
        NodeV<PK> n;
        float4 a = hi[o], b = c[o];
        n.F = {a.x, a.y}; n.Pp = {a.z, a.w};
        n.Fc = {b.x, b.y}; n.Pc = {b.z, b.w};
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
    Cx<T> DpS;       // (Dp_R + Dp_L)/2 = u~-averaged theta difference to the next row, minus the Hs part
    Cx<T> FC, PC;    // u~ = (h_R + h_L)/2 for Phi and Pi
    Cx<T> dFc, dPc;  // h_R - h_L for Phi and Pi
    __device__ __forceinline__ CRow mirror(T g) const {
        CRow r;
        r.Hs = g * Hs; r.DpS = g * DpS; r.FC = g * FC; r.PC = g * PC; r.dFc = g * dFc; r.dPc = g * dPc;
        return r;
    }
};

template <typename T>
struct CRing {
    CRow<T> a, b, c;  // rows jc-1, jc, jc+1 once full
    __device__ __forceinline__ void push(const CRow<T>& r) { a = b; b = c; c = r; }
};

template <typename T>
__device__ __forceinline__ void load_coefs(const T* tab, size_t pl, size_t o, bool ok, T* cf) {
#pragma unroll
    for (int k = 0; k < kNCoef; ++k) cf[k] = ok ? __ldg(tab + k * pl + o) : T(0);
}

// FP32 coefficients of one node from its radial table and its theta row (see RTab).
__device__ __forceinline__ void form_coefs(const RTab& t, const ThTab& h, float* cf) {
    float sig2 = fmaf(-t.aD, h.sin2, t.R2);
    float iS = __frcp_rn(sig2);
    float rs = rsqrtf(sig2);
    rs = rs * fmaf(-0.5f * sig2 * rs, rs, 1.5f);  // one Newton step on 1/sqrt
    float g = t.Rd * rs;
    float ctre = t.ctr * iS;
    float ctim = fmaf(t.ctc, h.cs, t.cti) * iS;
    cf[C_G] = g;
    cf[C_E1R] = -t.sdt * ctre;
    cf[C_E1I] = -t.sdt * ctim;
    float bbt = t.bb * h.sin2 * iS;
    cf[C_E2R] = fmaf(ctre, g, (t.pr - bbt) * iS);
    cf[C_E2I] = fmaf(ctim, g, t.pi * iS);
    float ws = t.Ds * iS;
    cf[C_EP] = ws * h.thp;
    cf[C_EM] = ws * h.thm;
    cf[C_E3R] = fmaf(-t.Ds, h.V, t.qr) * iS;
    cf[C_E3I] = t.qi * iS;
}

// The radial table of one column, held in registers for a whole work item (FP32 paths;
// empty for FP64, which reads 2D tables).
template <class P>
struct ColTab {
    RTab t;
    __device__ __forceinline__ void load(const RTab* tab, int i, bool ok) {
        if constexpr (sizeof(typename P::T) == 4) {
            if (ok) {
                const float4* q = (const float4*)(tab + i);
                float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), e = __ldg(q + 3);
                t = RTab{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, e.x, 0.f, 0.f, 0.f};
            } else {
                t = RTab{};
            }
        }
    }
};

// Coefficients of the predictor (half = true, node i+1/2) or the corrector (node i) at
// row j: read from the 2D FP64 tables, or formed in registers on the FP32 paths from
// the column's radial table and the row's theta table.
template <class P>
__device__ __forceinline__ void get_coefs(const InstDev& d, const ColTab<P>& col, bool half, int i,
                                          int j, bool ok, typename P::T* cf) {
    if constexpr (sizeof(typename P::T) == 8) {
        load_coefs((const double*)(half ? d.coef_h : d.coef_i), plane_elems(d),
                   (size_t)j * d.pitch + i, ok, cf);
    } else {
        const ThTab h = d.thtab[j];
        form_coefs(col.t, h, cf);
        if (!ok) {
#pragma unroll
            for (int k = 0; k < kNCoef; ++k) cf[k] = 0.f;
        }
    }
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

template <typename T>
__device__ __forceinline__ CRow<T> combine_lr(const HalfRec<T>& R) {
    HalfRec<T> L;
    L.Fb = shfl_up_c(R.Fb); L.Pb = shfl_up_c(R.Pb);
    L.dF = shfl_up_c(R.dF); L.dP = shfl_up_c(R.dP);
    L.Dp = shfl_up_c(R.Dp);
    L.hF = shfl_up_c(R.hF); L.hP = shfl_up_c(R.hP);
    CRow<T> c;
    c.Hs = Cx<T>::half_sum(R.hF, L.hF);
    c.DpS = Cx<T>::half_sum(R.Dp, L.Dp);
    c.FC = Cx<T>::half_sum(R.Fb, L.Fb) + c.Hs;
    c.PC = Cx<T>::half_sum(R.Pb, L.Pb) + Cx<T>::half_sum(R.hP, L.hP);
    c.dFc = Cx<T>::half_sum(R.dF, L.dF) + (R.hF - L.hF);
    c.dPc = Cx<T>::half_sum(R.dP, L.dP) + (R.hP - L.hP);
    return c;
}

// ---------------------------------------------------------------- source
__device__ __forceinline__ void source_factors(const InstDev& d, int64_t step, double2& sp,
                                               double2& sc) {
    double A = (d.src.amps != nullptr && step < d.src.n_amps) ? d.src.amps[step] : 1.0;
    double t = (double)step * d.dt;
    double s1, c1, s2, c2;
    sincos(d.src.omega * t + d.src.phase0, &s1, &c1);
    sincos(d.src.omega * (t + 0.5 * d.dt) + d.src.phase0, &s2, &c2);
    double hp = 0.5 * d.dt * A, hc = d.dt * A;
    sp = make_double2(hp * c1, -hp * s1);
    sc = make_double2(hc * c2, -hc * s2);
}

template <typename T>
__device__ __forceinline__ Cx<T> cmul_cast(double2 f, double2 p) {
    return {(T)(f.x * p.x - f.y * p.y), (T)(f.x * p.y + f.y * p.x)};
}

template <typename T>
__device__ __forceinline__ Cx<T> source_half(const SourceDev& s, double2 fac, int i, int j) {
    int a = i - s.h_lo, b = j - s.j_lo;
    if ((unsigned)a < (unsigned)s.nh && (unsigned)b < (unsigned)s.nj)
        return cmul_cast<T>(fac, s.P_half[(size_t)b * s.nh + a]);
    return Cx<T>::zero();
}

template <typename T>
__device__ __forceinline__ Cx<T> source_int(const SourceDev& s, double2 fac, int i, int j) {
    int a = i - s.i_lo, b = j - s.j_lo;
    if ((unsigned)a < (unsigned)s.ni && (unsigned)b < (unsigned)s.nj)
        return cmul_cast<T>(fac, s.P_int[(size_t)b * s.ni + a]);
    return Cx<T>::zero();
}

// Eq. (14) for row jc of the own column, store of u^{n+1}, and the waveform
// record of the input state (time level `step`) when this warp holds r*_ext.
template <class P>
__device__ __forceinline__ void corrector(const InstDev& d, const Planes<P>& in,
                                          const Planes<P>& out, const CRing<typename P::T>& ring,
                                          int jc, int i, bool out_ok, bool bnd, bool ex_warp,
                                          bool src_warp, const ColTab<P>& coli,
                                          typename P::T fdt, double2 sc_fac, int64_t step) {
    using T = typename P::T;
    using C = Cx<T>;
    const CRow<T>& a = ring.a;
    const CRow<T>& b = ring.b;
    const CRow<T>& c = ring.c;
    const bool col_ok = i < d.nr;
    C Dplus = b.DpS + (c.Hs - b.Hs);
    C Dminus = a.DpS + (b.Hs - a.Hs);
    const size_t o = (size_t)jc * d.pitch + i;
    T cf[kNCoef];
    get_coefs<P>(d, coli, false, i, jc, col_ok, cf);
    C src = C::zero();
    if (src_warp) src = source_int<T>(d.src, sc_fac, i, jc);
    C dPhi = rmac(rmac(C::zero(), -cf[C_G], b.dFc), fdt, b.PC);
    C dPi = rmac(src, cf[C_G], b.dPc);
    dPi = cmac(dPi, cf[C_E1R], cf[C_E1I], b.PC);
    dPi = cmac(dPi, cf[C_E2R], cf[C_E2I], b.dFc);
    dPi = rmac(dPi, cf[C_EP], Dplus);
    dPi = rmac(dPi, -cf[C_EM], Dminus);
    dPi = cmac(dPi, cf[C_E3R], cf[C_E3I], b.FC);
    NodeV<P> u = col_ok ? in.load(o) : NodeV<P>::zero();
    if (ex_warp) {
        double2 ph = u.phi64();
        double2 phn = make_double2(__shfl_down_sync(kFull, ph.x, 1), __shfl_down_sync(kFull, ph.y, 1));
        if (i == d.i_e) {
            double f = d.f_e;
            double2 w = make_double2((1.0 - f) * ph.x + f * phn.x, (1.0 - f) * ph.y + f * phn.y);
            d.wave[(size_t)(step % d.wave_cap) * d.nth + jc] = w;
            if (!isfinite(w.x) || !isfinite(w.y)) atomicOr(d.status, (unsigned)ST_NONFINITE);
        }
    }
    if (out_ok) {
        u.update(dPhi, dPi);
        out.store(o, u);
    } else if (bnd) {
        out.store(o, NodeV<P>::zero());
    }
}

}  // namespace teuk
