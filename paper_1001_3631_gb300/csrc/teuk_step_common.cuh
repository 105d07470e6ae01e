// teuk_step_common.cuh -- device building blocks of the Lax-Wendroff step kernels:
// precision policies, node loads/stores, the compensated update, the predictor
// (Eq. 13) and corrector (Eq. 14) bodies.  See teuk_step.cu for the scheme.
#pragma once
#include "teuk_df.cuh"
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
// Complex double-float values in paired instructions: the high parts (re, im) and the
// low parts (re, im) each form a register pair, and every step of the scalar
// double-float operation (teuk_df.cuh) runs on both components at once, with the same
// roundings, so the results equal the scalar code's.
struct DF2 { float2 hi, lo; };
__device__ __forceinline__ DF2 pk2(Cx<DF> a) {
    return {make_float2(a.re.hi, a.im.hi), make_float2(a.re.lo, a.im.lo)};
}
__device__ __forceinline__ Cx<DF> up2(DF2 v) { return {DF(v.hi.x, v.lo.x), DF(v.hi.y, v.lo.y)}; }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(bc(-1.0f), b, a); }   // exact product
__device__ __forceinline__ float2 p_neg(float2 a) { return __fmul2_rn(bc(-1.0f), a); }
// s + e = a + b exactly (per component)
__device__ __forceinline__ DF2 p_two_sum(float2 a, float2 b) {
    const float2 s = p_add(a, b);
    const float2 bb = p_sub(s, a);
    return {s, p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb))};
}
// s + e = a - b exactly (two_sum with -b written out)
__device__ __forceinline__ DF2 p_two_diff(float2 a, float2 b) {
    const float2 s = p_sub(a, b);
    const float2 bb = p_sub(s, a);
    return {s, p_sub(p_sub(a, p_sub(s, bb)), p_add(b, bb))};
}
__device__ __forceinline__ DF2 p_fast_two_sum(float2 a, float2 b) {
    const float2 s = p_add(a, b);
    return {s, p_sub(b, p_sub(s, a))};
}
__device__ __forceinline__ Cx<DF> operator+(Cx<DF> x, Cx<DF> y) {
    const DF2 X = pk2(x), Y = pk2(y);
    const DF2 S = p_two_sum(X.hi, Y.hi);
    return up2(p_fast_two_sum(S.hi, p_add(S.lo, p_add(X.lo, Y.lo))));
}
__device__ __forceinline__ Cx<DF> operator-(Cx<DF> x, Cx<DF> y) {
    const DF2 X = pk2(x), Y = pk2(y);
    const DF2 S = p_two_diff(X.hi, Y.hi);
    return up2(p_fast_two_sum(S.hi, p_add(S.lo, p_sub(X.lo, Y.lo))));
}
__device__ __forceinline__ Cx<DF> neg(Cx<DF> a) {
    const DF2 A = pk2(a);
    return up2({p_neg(A.hi), p_neg(A.lo)});
}
// a * b + c per component, a given as pairs (hi, lo): the double-float tfma
__device__ __forceinline__ DF2 p_tfma(DF2 A, DF2 B, DF2 C) {
    const float2 p = __fmul2_rn(A.hi, B.hi);
    float2 e = __ffma2_rn(A.hi, B.hi, p_neg(p));
    e = __ffma2_rn(A.hi, B.lo, e);
    e = __ffma2_rn(A.lo, B.hi, e);
    const DF2 S = p_two_sum(p, C.hi);
    return p_fast_two_sum(S.hi, p_add(S.lo, p_add(e, C.lo)));
}
__device__ __forceinline__ DF2 bc2(DF s) { return {bc(s.hi), bc(s.lo)}; }
__device__ __forceinline__ Cx<DF> operator*(DF s, Cx<DF> a) {
    const DF2 S = bc2(s), A = pk2(a);
    const float2 p = __fmul2_rn(S.hi, A.hi);
    float2 e = __ffma2_rn(S.hi, A.hi, p_neg(p));
    e = __ffma2_rn(S.hi, A.lo, e);
    e = __ffma2_rn(S.lo, A.hi, e);
    return up2(p_fast_two_sum(p, e));
}
__device__ __forceinline__ Cx<DF> rmac(Cx<DF> acc, DF s, Cx<DF> z) {
    return up2(p_tfma(bc2(s), pk2(z), pk2(acc)));
}
// same order as the generic cmac: the ci terms first, then the cr terms
__device__ __forceinline__ Cx<DF> cmac(Cx<DF> acc, DF cr, DF ci, Cx<DF> z) {
    const DF2 Z = pk2(z);
    const DF2 Zs = {make_float2(Z.hi.y, Z.hi.x), make_float2(Z.lo.y, Z.lo.x)};   // (im, re)
    const DF2 Ci = {make_float2(-ci.hi, ci.hi), make_float2(-ci.lo, ci.lo)};
    return up2(p_tfma(bc2(cr), Z, p_tfma(Ci, Zs, pk2(acc))));
}
template <>
__device__ __forceinline__ Cx<DF> Cx<DF>::half_sum(Cx<DF> a, Cx<DF> b) {
    const DF2 s = pk2(a + b);
    return up2({__fmul2_rn(bc(0.5f), s.hi), __fmul2_rn(bc(0.5f), s.lo)});
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
// kind: the teuk_precision value; planes: 16-byte planes per state buffer (the layout
// in teuk_internal.cuh); blocks256: resident blocks per SM that the register budget of
// the step kernel for columns of up to 256 rows aims at (two: at three the FP32 paths
// fit in 80 registers but run no faster, being issue-bound)
enum PrecKind { kFP64 = 0, kFP32 = 1, kKahan = 2, kDF = 3 };
struct P64 {
    using T = double;
    static constexpr bool kahan = false;
    static constexpr int kind = kFP64, planes = 2, blocks256 = 2;
};
struct P32 {
    using T = float;
    static constexpr bool kahan = false;
    static constexpr int kind = kFP32, planes = 1, blocks256 = 2;
};
struct PK {
    using T = float;
    static constexpr bool kahan = true;
    static constexpr int kind = kKahan, planes = 2, blocks256 = 2;
};
// FP64-equivalent: double-float state, coefficients and arithmetic on the FP32 units
struct PD {
    using T = DF;
    static constexpr bool kahan = false;
    static constexpr int kind = kDF, planes = 2, blocks256 = 2;
};
// the FP32 paths that form their coefficients from 1D tables
template <class P>
__host__ __device__ constexpr bool uses_1d_tables() { return P::kind == kFP32 || P::kind == kKahan; }

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
    // Split theta differences of Phi at this node from the rows above (a, factor ga)
    // and below (b, factor gb): d2 = ga a - 2 this + gb b and d1 = ga a - gb b.  For
    // compensated pairs the hi differences (exact for neighbouring values within a
    // factor of two) and the c differences are combined first, so d2 and d1 round
    // relative to their own size, not to that of the first differences.
    __device__ __forceinline__ void theta_split(T ga, const NodeV& a, T gb, const NodeV& b,
                                                Cx<T>& d2, Cx<T>& d1) const {
        const Cx<T> hp = rmac(neg(F), ga, a.F);   // ga a - this
        const Cx<T> hm = rmac(F, -gb, b.F);       // this - gb b
        if constexpr (P::kahan) {
            const Cx<T> cp = rmac(neg(Fc), ga, a.Fc);
            const Cx<T> cm = rmac(Fc, -gb, b.Fc);
            d2 = (hp - hm) - (cp - cm);
            d1 = (hp + hm) - (cp + cm);
        } else {
            d2 = hp - hm;
            d1 = hp + hm;
        }
    }
    __device__ __forceinline__ Cx<T> dpi(const NodeV& o) const {
        if constexpr (P::kahan) return (Pp - o.Pp) - (Pc - o.Pc);
        else return Pp - o.Pp;
    }
    __device__ __forceinline__ double2 phi64() const {
        double v[4];
        v64(v);
        return make_double2(v[0], v[1]);
    }
    // {Phi_R, Phi_I, Pi_R, Pi_I} as FP64
    __device__ __forceinline__ void v64(double* v) const {
        if constexpr (P::kind == kDF) {
            v[0] = F.re.to_double(); v[1] = F.im.to_double();
            v[2] = Pp.re.to_double(); v[3] = Pp.im.to_double();
        } else if constexpr (P::kahan) {
            v[0] = (double)F.re - (double)Fc.re; v[1] = (double)F.im - (double)Fc.im;
            v[2] = (double)Pp.re - (double)Pc.re; v[3] = (double)Pp.im - (double)Pc.im;
        } else {
            v[0] = (double)F.re; v[1] = (double)F.im; v[2] = (double)Pp.re; v[3] = (double)Pp.im;
        }
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

template <> struct Planes<PD> {
    float4* hi; float4* lo;   // {Phi, Pi} high parts, low parts
    __device__ __forceinline__ static Planes of(const InstDev& d, int b) {
        return {(float4*)d.buf[b][0], (float4*)d.buf[b][1]};
    }
    __device__ __forceinline__ static Planes at(void* base, unsigned stride) {
        return {(float4*)base, (float4*)base + stride};
    }
    __device__ __forceinline__ NodeV<PD> load(size_t o) const {
        NodeV<PD> n;
        const float4 a = hi[o], b = lo[o];
        n.F = {DF(a.x, b.x), DF(a.y, b.y)};
        n.Pp = {DF(a.z, b.z), DF(a.w, b.w)};
        n.Fc = n.Pc = Cx<DF>::zero();
        return n;
    }
    __device__ __forceinline__ NodeV<PD> load_phi(size_t o) const {
        NodeV<PD> n = NodeV<PD>::zero();
        const float2 a = *(const float2*)(hi + o), b = *(const float2*)(lo + o);
        n.F = {DF(a.x, b.x), DF(a.y, b.y)};
        return n;
    }
    __device__ __forceinline__ void store(size_t o, const NodeV<PD>& n) const {
        hi[o] = make_float4(n.F.re.hi, n.F.im.hi, n.Pp.re.hi, n.Pp.im.hi);
        lo[o] = make_float4(n.F.re.lo, n.F.im.lo, n.Pp.re.lo, n.Pp.im.lo);
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
        h.Fb = Cx<T>::half_sum(own.F, nb.F);
        h.Pb = Cx<T>::half_sum(own.Pp, nb.Pp);
    }
    h.dF = nb.dphi(own);
    h.dP = nb.dpi(own);
    return h;
}

// Angular term of S_Pi, w Theta[F] - w V F (the V part sits in E3), in one of two forms:
//   expanded (FP64, double-float): ep (F_{j+1} - F_j) - em (F_j - F_{j-1}),
//   split (FP32 paths):            A (F_{j+1} - 2 F_j + F_{j-1}) + B (F_{j+1} - F_{j-1}),
//   A = s dt w / dth^2, B = s dt w cot / (2 dth)  (ep = A + B, em = A - B).
// The two are the same operator.  In FP32 the split form keeps the large coefficient
// A on the second difference, which is formed from the compensated pairs to its own
// relative accuracy; the expanded form would round ep and em separately and apply
// them to first differences, an error of order A times the first difference that the
// long-run growth of the angular modes then amplifies.
template <class P>
__host__ __device__ constexpr bool split_angular() { return P::kind == kFP32 || P::kind == kKahan; }

// Predictor output at one half node, plus the inputs the corrector needs from it.
// Expanded form: Dp = Fb(j+1) - Fb(j) (D1 unused); split form: Dp = Fb(j+1) - 2 Fb(j) +
// Fb(j-1), D1 = Fb(j+1) - Fb(j-1).
template <typename T>
struct HalfRec { Cx<T> Fb, Pb, dF, dP, Dp, D1, hF, hP; };

// Corrector inputs of one row, combined from the half nodes R = i+1/2 and L = i-1/2.
template <typename T>
struct CRow {
    Cx<T> Hs;        // (dh_Phi_R + dh_Phi_L)/2
    Cx<T> DpS;       // (Dp_R + Dp_L)/2
    Cx<T> D1S;       // (D1_R + D1_L)/2 (split form)
    Cx<T> FC, PC;    // u~ = (h_R + h_L)/2 for Phi and Pi
    Cx<T> dFc, dPc;  // h_R - h_L for Phi and Pi
};

template <typename T, bool kSplit>
__device__ __forceinline__ CRow<T> combine_lr(const HalfRec<T>& R, const HalfRec<T>& L) {
    CRow<T> c;
    c.Hs = Cx<T>::half_sum(R.hF, L.hF);
    c.DpS = Cx<T>::half_sum(R.Dp, L.Dp);
    if constexpr (kSplit) c.D1S = Cx<T>::half_sum(R.D1, L.D1);
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
struct ThPair { float2 sin2, cs, V, i2, i1; };
template <class P>
struct RowTab {
    ThPair t;
    __device__ __forceinline__ void load(const ThTab* tab, int j, bool ok) {
        if constexpr (uses_1d_tables<P>()) {
            const ThTab h = ok ? tab[j] : ThTab{};
            t = ThPair{bc(h.sin2), bc(h.cs), bc(h.V), bc(h.i2), bc(h.i1)};
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
    cf[C_EP] = __fmul2_rn(ws, h.i2);   // A (split angular form)
    cf[C_EM] = __fmul2_rn(ws, h.i1);   // B
    cf[C_E3R] = __fmul2_rn(__ffma2_rn(t.nDs, h.V, t.qr), iS);
    cf[C_E3I] = __fmul2_rn(t.qi, iS);
}

// FP64 coefficients of the predictor (half = true, node i+1/2) or the corrector (node i)
// at row j, from the 2D tables.
__device__ __forceinline__ void coefs64(const InstDev& d, bool half, int i, int j, double* cf) {
    load_coefs((const double*)(half ? d.coef_h : d.coef_i), plane_elems(d), node_index(d, i, j), cf);
}
// Double-float coefficients (FP64-equivalent path), from its 2D tables of (hi, lo) pairs.
__device__ __forceinline__ void coefs_df(const InstDev& d, bool half, int i, int j, DF* cf) {
    const float2* tab = (const float2*)(half ? d.coef_h : d.coef_i);
    const size_t pl = plane_elems(d), o = node_index(d, i, j);
#pragma unroll
    for (int k = 0; k < kNCoef; ++k) {
        const float2 v = __ldg(tab + k * pl + o);
        cf[k] = DF(v.x, v.y);
    }
}

// Eq. (13) at the own half node, as an increment on the averaged state.  Dp, Dm: the
// theta differences of the averaged state in the angular form of kSplit (expanded:
// forward and backward differences; split: second and two-cell differences).
template <typename T, bool kSplit>
__device__ __forceinline__ HalfRec<T> predictor(const Half<T>& h, Cx<T> Dp, Cx<T> Dm, const T* cf,
                                                T hdt, Cx<T> src) {
    HalfRec<T> r;
    r.Fb = h.Fb; r.Pb = h.Pb; r.dF = h.dF; r.dP = h.dP; r.Dp = Dp; r.D1 = Dm;
    r.hF = rmac(rmac(Cx<T>::zero(), -cf[C_G], h.dF), hdt, h.Pb);
    Cx<T> a = rmac(src, cf[C_G], h.dP);
    a = cmac(a, cf[C_E1R], cf[C_E1I], h.Pb);
    a = cmac(a, cf[C_E2R], cf[C_E2I], h.dF);
    if constexpr (kSplit) {
        a = rmac(a, cf[C_EP], Dp);
        a = rmac(a, cf[C_EM], Dm);
    } else {
        a = rmac(a, cf[C_EP], Dp);
        a = rmac(a, -cf[C_EM], Dm);
    }
    a = cmac(a, cf[C_E3R], cf[C_E3I], h.Fb);
    r.hP = a;
    return r;
}

// ---------------------------------------------------------------- extraction
// Waveform record between the nodes i_e (a) and i_e + 1 (b): (1 - f) a + f b, written with
// explicit roundings so that every kernel that records a level rounds it the same way.
__device__ __forceinline__ double2 wave_lerp(double2 a, double2 b, double f) {
    const double g = 1.0 - f;
    return make_double2(__fma_rn(f, b.x, __dmul_rn(g, a.x)), __fma_rn(f, b.y, __dmul_rn(g, a.y)));
}

// ---------------------------------------------------------------- corrector
// Exchange entry of one row for the corrector's theta neighbours: {Hs, DpS} (4 values of
// T at e; the split form uses Hs alone).  Row j sits at entry j + 1 of its column's
// buffer; entries 0 and n_theta + 1 hold the ghost rows of the pole rule:
// row nth Hs = g Hs(nth-1); row -1 Hs = g Hs(0) and DpS = (Dp_R(-1) + Dp_L(-1))/2 =
// (1 - g) (Fb_R + Fb_L)(0)/2.
template <class P>
__device__ __forceinline__ void xput(typename P::T* e, Cx<typename P::T> a, Cx<typename P::T> b) {
    if constexpr (P::kind == kDF) {
        ((float4*)e)[0] = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
        ((float4*)e)[1] = make_float4(b.re.hi, b.re.lo, b.im.hi, b.im.lo);
    } else if constexpr (sizeof(typename P::T) == 4) {
        *(float4*)e = make_float4(a.re, a.im, b.re, b.im);
    } else {
        ((double2*)e)[0] = make_double2(a.re, a.im);
        ((double2*)e)[1] = make_double2(b.re, b.im);
    }
}

// Publish this row's entry (xb: the column's buffer, mine = xb + 4 (j + 1)) and, for the
// pole rows, the ghost entries.
template <class P, bool kSplit>
__device__ __forceinline__ void xpublish(typename P::T* xb, typename P::T* mine, const CRow<typename P::T>& row,
                                         const HalfRec<typename P::T>& Rh, const HalfRec<typename P::T>& Lh,
                                         typename P::T g, bool row_ok, bool top, bool bot) {
    using T = typename P::T;
    using C = Cx<T>;
    if constexpr (kSplit) {
        if (row_ok) *(float2*)mine = make_float2(row.Hs.re, row.Hs.im);
        if (top) *(float2*)(mine + 4) = make_float2(g * row.Hs.re, g * row.Hs.im);
        if (bot) *(float2*)xb = make_float2(g * row.Hs.re, g * row.Hs.im);
    } else {
        if (row_ok) xput<P>(mine, row.Hs, row.DpS);
        if (top) xput<P>(mine + 4, g * row.Hs, C::zero());
        if (bot) xput<P>(xb, g * row.Hs, (T(1) - g) * C::half_sum(Rh.Fb, Lh.Fb));
    }
}

// Read the entries of the rows above and below (after the barrier that follows xpublish).
template <class P, bool kSplit>
__device__ __forceinline__ void xread(const typename P::T* mine, Cx<typename P::T>& Hs_p,
                                      Cx<typename P::T>& Hs_m, Cx<typename P::T>& DpS_m) {
    if constexpr (kSplit) {
        const float2 a = *(const float2*)(mine + 4), b = *(const float2*)(mine - 4);
        Hs_p = {a.x, a.y};
        Hs_m = {b.x, b.y};
    } else if constexpr (P::kind == kDF) {
        const float4 a = *(const float4*)(mine + 4);
        const float4 b0 = ((const float4*)(mine - 4))[0], b1 = ((const float4*)(mine - 4))[1];
        Hs_p = {DF(a.x, a.y), DF(a.z, a.w)};
        Hs_m = {DF(b0.x, b0.y), DF(b0.z, b0.w)};
        DpS_m = {DF(b1.x, b1.y), DF(b1.z, b1.w)};
    } else if constexpr (sizeof(typename P::T) == 4) {
        const float2 a = *(const float2*)(mine + 4);
        const float4 b = *(const float4*)(mine - 4);
        Hs_p = {a.x, a.y};
        Hs_m = {b.x, b.y};
        DpS_m = {b.z, b.w};
    } else {
        const double2 a = *(const double2*)(mine + 4);
        const double2 b0 = ((const double2*)(mine - 4))[0], b1 = ((const double2*)(mine - 4))[1];
        Hs_p = {a.x, a.y};
        Hs_m = {b0.x, b0.y};
        DpS_m = {b1.x, b1.y};
    }
}

// Eq. (14) at one node as increments (dPhi, dPi) from the row's combined half-node values,
// the theta neighbours' exchange entries, the node's coefficients cf and source term.
template <class P, bool kSplit>
__device__ __forceinline__ void corrector_incr(const CRow<typename P::T>& row, Cx<typename P::T> Hs_p,
                                               Cx<typename P::T> Hs_m, Cx<typename P::T> DpS_m,
                                               const typename P::T* cf, typename P::T fdt,
                                               Cx<typename P::T> srcc, Cx<typename P::T>& dPhi,
                                               Cx<typename P::T>& dPi) {
    using C = Cx<typename P::T>;
    // expanded: Dplus = u~(j+1) - u~(j), Dminus = u~(j) - u~(j-1) of the corrector's
    // averaged state u~ = (h_R + h_L)/2; split: its second and two-cell differences
    C Dplus, Dminus;
    if constexpr (kSplit) {
        Dplus = row.DpS + ((Hs_p - row.Hs) - (row.Hs - Hs_m));
        Dminus = row.D1S + (Hs_p - Hs_m);
    } else {
        Dplus = row.DpS + (Hs_p - row.Hs);
        Dminus = DpS_m + (row.Hs - Hs_m);
    }
    dPhi = rmac(rmac(C::zero(), -cf[C_G], row.dFc), fdt, row.PC);
    dPi = rmac(srcc, cf[C_G], row.dPc);
    dPi = cmac(dPi, cf[C_E1R], cf[C_E1I], row.PC);
    dPi = cmac(dPi, cf[C_E2R], cf[C_E2I], row.dFc);
    if constexpr (kSplit) {
        dPi = rmac(dPi, cf[C_EP], Dplus);
        dPi = rmac(dPi, cf[C_EM], Dminus);
    } else {
        dPi = rmac(dPi, cf[C_EP], Dplus);
        dPi = rmac(dPi, -cf[C_EM], Dminus);
    }
    dPi = cmac(dPi, cf[C_E3R], cf[C_E3I], row.FC);
}

// ---------------------------------------------------------------- source
// dt_sub A_n e^{-i (omega t + phase0)} at t = t_n + off * dt: the predictor's factor
// (off = 0, dt_sub = dt/2) or the corrector's (off = 1/2, dt_sub = dt); for a moving
// particle dt_sub A e^{-i m phi_p} of the step's sample (the Gaussian is tabulated)
template <bool kMov>
__device__ __forceinline__ double2 source_factor(const InstDev& d, int64_t step, double off,
                                                 double dt_sub) {
    if constexpr (kMov) {
        if (d.src.moving) {   // sample 2n (off = 0) or 2n + 1 (off = 1/2) of a sampled path
            if (step >= d.src.n_traj) return make_double2(0.0, 0.0);
            const double2 A = d.src.amp[2 * step + (off == 0.0 ? 0 : 1)];
            return make_double2(dt_sub * A.x, dt_sub * A.y);
        }
    }
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
struct DFC { DF x, y; };   // complex double-float as stored: x.hi, x.lo, y.hi, y.lo
template <> struct V2T<DF> { using V = DFC; };

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
