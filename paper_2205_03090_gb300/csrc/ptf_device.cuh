// ptf_device.cuh -- per-thread FP64 building blocks of the flash (sm_103a).
//
// One mixture per thread; NC (number of components) is a template parameter
// so per-component vectors live in registers.  Everything here is FP64
// except the FP32 starting guess of the cubic root, which FP64 Halley
// iterations then refine to full precision.
//
// Paper references (arXiv 2205.03090): SRK EOS and mixing rules (Appendix A,
// Eqs. mixing_rule, cubic_Z, halley, lnphi), Wilson K (Eq. wilson),
// Rachford-Rice (Eq. RR, Appendix C, Eq. RR_helper), trust-region method
// (Appendix B, Eqs. tr_sa, analysis_grad/hess, newton_splitter,
// split_grad/hess), DEM (Sec. 2.2.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ptf_logtab.cuh"
#include "ptf_exptab.cuh"

namespace ptf {

// ---------------------------------------------------------------------------
// Constants printed in the paper and the method's controls
// ---------------------------------------------------------------------------
constexpr double kOmegaA = 0.42748;   // Eq. a_i
constexpr double kOmegaB = 0.08664;   // Eq. b_i
constexpr double kWilson = 5.373;     // Eq. wilson
constexpr double kTolStab = 1e-6;     // Sec. 2.2.1, Appendix B.1
constexpr double kTolSplitTR = 1e-8;  // Appendix B.2
// Fugacity residual at which a split stops: 2 % below the 1e-10 target, so
// that the target still holds when another FP64 implementation re-evaluates
// the point (rounding moves the residual by ~1e-15).
constexpr double kTolFug = 0.98e-10;
constexpr int kSSStab = 9;            // Alg. 2
constexpr int kTRStab = 20;           // Alg. 2
constexpr int kSSSplit = 9;           // Sec. 2.2.2
// The paper gives no cap for the split trust region (its Table 4 run needed
// at most 13 iterations); 60 lets the slow runs near three-phase conditions
// converge (the slowest seen needed 33 iterations with the polish).
constexpr int kTRSplit = 60;
constexpr int kNewtonPolish = 10;     // Newton steps after a split TR run
constexpr int kPrecheck = 3;          // Sec. 2.2.3
constexpr double kEpsNeg = 1e-10;     // "negative" tm / tpd / Delta G
constexpr double kTrivialLnK = 1e-6;  // split collapsed to K = 1
// A split trust-region iterate with theta this close to 0 or 1 has collapsed
// onto one phase without converging (each fraction-to-boundary step then moves
// theta some six decades further): the run stops there, single phase, not
// converged.
constexpr double kCollapseTheta = 1e-10;
constexpr double kPredTrust = 1e-12;  // ratio test trusted above this
// Learned form: a split started from the initializer's K keeps its result only
// if its converged ln K lie within this distance of the network's prediction
// (farther away, the split went to a stationary point other than the one the
// network was trained on, and the plain method redoes the mixture).
constexpr double kNNLnKDev = 0.3;

// Tolerances and iteration caps of one call (ptflash_options; the defaults
// above).  Part of the workspace descriptor, a kernel parameter, so every
// read is a uniform constant-bank load.
struct Ctl {
    int ss_stab = kSSStab, tr_stab = kTRStab, ss_split = kSSSplit, tr_split = kTRSplit, polish = kNewtonPolish;
    double tol_stab = kTolStab, tol_split_tr = kTolSplitTR, tol_fug = kTolFug;
    double nn_lnk_dev = kNNLnKDev;  // learned form: accepted max |ln K - ln K_net| of a network-started split
    // trust-region lanes per run: 0 one lane per run until the queue drains,
    // then several lanes per run; 1 one lane throughout; 2 several lanes
    // throughout (the results are the same bit for bit in every mode)
    int tr_coop = 0;
};

// status bits (same values as documented in include/ptflash.h)
constexpr int ST_PRECHECK_UNSTABLE = 1;
constexpr int ST_STAB_RUN = 2;
constexpr int ST_STAB_TR = 4;
constexpr int ST_SPLIT_TR = 8;
constexpr int ST_MAXITER = 16;
constexpr int ST_COLLAPSE = 32;
constexpr int ST_NONFINITE = 64;
constexpr int ST_NN_STABLE = 128;
constexpr int ST_NN_UNSTABLE = 256;
constexpr int ST_NN_INIT = 512;
constexpr int ST_NN_REJECT = 1024;

// Component table, passed by value as a kernel parameter (constant bank:
// every access is a uniform broadcast).
template <int NC>
struct Comp {
    double kk[NC * NC];  // 1 - k_ij
    double Tc[NC], Pc[NC], lnPc[NC], mi[NC], wc[NC];  // wc = 5.373 (1 + omega)
    double rsTc[NC], sOmA[NC], OmB[NC];  // 1 / sqrt(Tc), sqrt(0.42748 / Pc), 0.08664 / Pc
    float kkf[NC * NC];  // 1 - k_ij in FP32 (the FP32 stability pre-iteration)
};

// ---------------------------------------------------------------------------
// Natural logarithm for positive normal doubles by a table-driven reduction
// (P. T. P. Tang, ACM TOMS 16 (1990) 378): x = 2^e m, m in [0.75, 1.5),
// nearest breakpoint F = 0.75 + j/128, r = (m - F)/F with |r| <= 1/192, and
// ln x = e ln 2 + ln F + ln(1 + r), ln(1 + r) by its Taylor series to r^7
// (truncation below 1e-19).  Exponent, mantissa, index and F come from
// integer operations; m - F is exact (Sterbenz).  About 12 FP64 operations
// against ~36 FP64 pipe slots of the library log on this GPU.  Zero,
// negative, subnormal, infinite and NaN inputs go to the library log.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double log_fast(double x) {
    const long long b = __double_as_longlong(x);
    if ((unsigned long long)(b - 0x0010000000000000LL) >= 0x7fe0000000000000ULL) return log(x);
    long long e = (b >> 52) - 1023;
    const long long frac = b & 0x000fffffffffffffLL;
    long long mb, fb;
    int j;
    if (frac >= 0x0008000000000000LL) {  // m >= 1.5: use m / 2 in [0.75, 1)
        e += 1;
        mb = frac | 0x3fe0000000000000LL;
        j = (int)((frac + (1LL << 45)) >> 46) - 32;                  // round((m/2 - 0.75) 128)
        fb = 0x3fe0000000000000LL + ((long long)(32 + j) << 46);     // F = (1.5 + j/64) / 2
    } else {                            // m in [1, 1.5)
        mb = frac | 0x3ff0000000000000LL;
        j = 32 + (int)((frac + (1LL << 44)) >> 45);                  // round((m - 0.75) 128)
        fb = 0x3ff0000000000000LL + ((long long)(j - 32) << 45);     // F = 1 + (j - 32)/128
    }
    const double m = __longlong_as_double(mb), F = __longlong_as_double(fb);
    const double invF = __ldg(&kLogTab[j][0]), lnF = __ldg(&kLogTab[j][1]);
    const double r = (m - F) * invF;
    double t = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    t = fma(t, r, 0.2);
    t = fma(t, r, -0.25);
    t = fma(t, r, 1.0 / 3.0);
    t = fma(t, r, -0.5);
    const double l1p = fma(t, r * r, r);
    const double ed = __longlong_as_double(0x4338000000000000LL + e) - 6755399441055744.0;  // (double)e
    return fma(ed, 0.6931471805599453, lnF + l1p);
}

// ---------------------------------------------------------------------------
// Exponential for |x| < 708 by the table-driven method of P. T. P. Tang (ACM
// TOMS 15 (1989) 144): n = rint(64 x / ln 2) = 64 m + j, r = x - n ln2/64
// (two-part constant, |r| <= ln2/128), e^x = 2^m 2^(j/64) (1 + p(r)) with
// p(r) = e^r - 1 by its Taylor polynomial to r^6 (truncation below 3e-20).
// About 12 FP64 operations; outside the range (overflow, underflow, NaN) the
// library exp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double exp_fast(double x) {
    if (!(fabs(x) < 708.0)) return exp(x);
    const double shifter = 6755399441055744.0;  // 1.5 * 2^52: rint into the low bits
    const double t = fma(x, kExpInvL, shifter);
    const int n = (int)__double2loint(t);
    const double nf = t - shifter;
    double r = fma(-nf, kExpL1, x);
    r = fma(-nf, kExpL2, r);
    double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(q, r * r, r);
    const double T = __ldg(&kExpTab[n & 63]);
    const double v = fma(T, p, T);
    // times 2^m, m = n >> 6 (floor): add m to the exponent field
    return __longlong_as_double(__double_as_longlong(v) + ((long long)(n >> 6) << 52));
}

// Per-mixture EOS constants: sqrt(A_i) and B_i (reduced, R cancels).
template <int NC>
struct Mix {
    double sA[NC], B[NC];
};

// Appendix A: A_i = 0.42748 alpha_i (P/Pc)(Tc/T)^2, B_i = 0.08664 (P/Pc)(Tc/T),
// alpha_i = [1 + m_i (1 - sqrt(T/Tc))]^2.
// The component factors 1/sqrt(Tc_i), sqrt(0.42748/Pc_i) and 0.08664/Pc_i are
// in the table, so a mixture takes one division and two square roots for all
// its components: sqrt(A_i) = sqrt(0.42748/Pc_i) sqrt(P) |a_i| Tc_i / T with
// a_i = 1 + m_i (1 - sqrt(T) / sqrt(Tc_i)), and B_i = (0.08664/Pc_i) P Tc_i / T.
template <int NC>
__device__ __forceinline__ void mix_init(const Comp<NC>& cp, double P, double T, Mix<NC>& mx) {
    const double invT = 1.0 / T, sT = sqrt(T);
    const double sPT = sqrt(P) * invT, PT = P * invT;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double a = fma(cp.mi[i], fma(-sT, cp.rsTc[i], 1.0), 1.0);
        mx.sA[i] = cp.sOmA[i] * sPT * fabs(a) * cp.Tc[i];
        mx.B[i] = cp.OmB[i] * PT * cp.Tc[i];
    }
}

// Eq. wilson
template <int NC>
__device__ __forceinline__ void wilson(const Comp<NC>& cp, double P, double T, double* lnK) {
    double lnP = log_fast(P), invT = 1.0 / T;
#pragma unroll
    for (int i = 0; i < NC; i++) lnK[i] = cp.lnPc[i] - lnP + cp.wc[i] * (1.0 - cp.Tc[i] * invT);
}

// ---------------------------------------------------------------------------
// Cubic (Eq. cubic_Z) f(Z) = Z^3 - Z^2 + r1 Z - r0, r1 = A - B - B^2, r0 = AB.
// f(B) = -2B^2 < 0 and f(1+B) = A > 0, so (B, 1+B] holds a sign change and
// every admissible root (Z > B) lies in it.  The number of real roots follows
// from the values of f at its critical points.  One root is found by Halley
// iterations (Eq. halley) kept inside the sign-change bracket (bisection when
// a step leaves it, so the iteration cannot stall at an extremum): an FP32
// run seeds the FP64 run.  The FP64 run stops after a Halley step below 2e-6
// relative: Halley's cubic convergence leaves an error of order (2e-6)^3,
// far below what the paper's 1e-8 step criterion (Appendix A) guarantees.
// With three real roots, deflation (Appendix A) gives the other two.  Among
// admissible roots the smallest and the largest are compared by the residual
// Gibbs energy gbar(Z) = Z - 1 - ln(Z - B) - (A/B) ln(1 + B/Z).  The chosen
// root gets one FP64 Newton polish and its FP64 logarithms.
//
// Two decisions may be taken in FP32, each only where a bound on its FP32
// rounding error proves that FP64 takes the same one (u = 2^-24):
//  - the root count, from the signs of f at its critical points zm, zp (they
//    exist for r1 < 1/3).  Horner's rule on z < 1 from r1, r0 rounded to
//    FP32 is off by at most about 3u (z^3 + z^2 + |r1| z + r0) < 3u (3 + r0);
//    zm and zp are off by O(u / sqrt(4 - 12 r1)), which moves f only at second
//    order (f' vanishes there), so FP32 decides where 4 - 12 r1 > 1e-5 and
//    both |f| exceed 1e-5 (1 + r0), some 25 times the bound;
//  - the root choice, from the sign of gbar(zl) - gbar(zv).  zl - zv, zl - B,
//    zv - B, B/zl and B/zv are formed in FP64 (so no cancellation happens in
//    FP32) and rounded once; logf and log1pf then err by at most about one
//    FP32 ulp of their results, so each of the five terms t_k of the
//    difference is off by at most about 4u |t_k| + u, and FP32 decides where
//    the difference exceeds 1e-5 (1 + sum |t_k|), some 40 times the bound.
// Everywhere else both decisions are FP64.
// ---------------------------------------------------------------------------
struct Root {
    double Z, lzb, L;  // chosen root, ln(Z - B), ln(1 + B/Z)
};

__device__ __forceinline__ double cub_f(double Z, double r1, double r0) { return fma(fma(Z - 1.0, Z, r1), Z, -r0); }
__device__ __forceinline__ double cub_df(double Z, double r1) { return fma(fma(3.0, Z, -2.0), Z, r1); }
__device__ __forceinline__ double cub_polish(double Z, double r1, double r0) {
    const double d = cub_df(Z, r1);
    return d != 0.0 ? Z - cub_f(Z, r1, r0) / d : Z;
}

__device__ __forceinline__ Root cubic_select(double A, double B) {
    const double r1 = A - B * (1.0 + B), r0 = A * B;
    // real-root count from the critical points of f (local max zm, local min
    // zp), in FP32 where the error bound above allows, else in FP64
    bool three = false;
    const float r1f = (float)r1, r0f = (float)r0;
    const float dcf = fmaf(-12.0f, r1f, 4.0f);
    if (dcf > -1e-5f) {
        bool decided = false;
        if (dcf > 1e-5f) {
            const float sqf = sqrtf(dcf);
            const float zmf = (2.0f - sqf) * (1.0f / 6.0f), zpf = (2.0f + sqf) * (1.0f / 6.0f);
            const float fm = fmaf(fmaf(zmf - 1.0f, zmf, r1f), zmf, -r0f);
            const float fpv = fmaf(fmaf(zpf - 1.0f, zpf, r1f), zpf, -r0f);
            const float tau = 1e-5f * (1.0f + fabsf(r0f));
            if (fabsf(fm) > tau && fabsf(fpv) > tau) {
                three = fm > 0.0f && fpv < 0.0f;
                decided = true;
            }
        }
        if (!decided) {
            const double dcrit = 4.0 - 12.0 * r1;
            if (dcrit > 0.0) {
                const double sq = sqrt(dcrit);
                const double fm = cub_f((2.0 - sq) * (1.0 / 6.0), r1, r0), fpv = cub_f((2.0 + sq) * (1.0 / 6.0), r1, r0);
                three = !(fm < 0.0) && !(fpv > 0.0);
            }
        }
    }
    // FP32 seed: bracketed Halley on (B, 1 + B]
    float lof = (float)B, hif = 1.0f + (float)B, zf = hif;
    {
#pragma unroll 1
        for (int it = 0; it < 40; it++) {
            float f = fmaf(fmaf(zf - 1.0f, zf, r1f), zf, -r0f);
            if (f < 0.0f) lof = zf; else hif = zf;
            float fp = fmaf(fmaf(3.0f, zf, -2.0f), zf, r1f);
            float fpp = fmaf(6.0f, zf, -2.0f);
            float zn = zf - 2.0f * f * fp / (2.0f * fp * fp - f * fpp);
            if (fabsf(zn - zf) <= 1e-6f * zf) {  // converged: accept before any bracket test
                zf = zn;
                break;
            }
            if (!(zn > lof && zn < hif)) zn = 0.5f * (lof + hif);
            zf = zn;
        }
    }
    // FP64 bracketed Halley from the seed
    double lo = B, hi = 1.0 + B, z0 = (double)zf;
    if (!(z0 > lo && z0 < hi)) z0 = 0.5 * (lo + hi);
#pragma unroll 1
    for (int it = 0; it < 100; it++) {
        double f = cub_f(z0, r1, r0);
        if (f < 0.0) lo = z0; else if (f > 0.0) hi = z0; else break;
        double fp = cub_df(z0, r1);
        double fpp = fma(6.0, z0, -2.0);
        double zn = z0 - 2.0 * f * fp / (2.0 * fp * fp - f * fpp);
        if (fabs(zn - z0) <= 2e-6 * fabs(zn)) {  // converged: accept before any bracket test
            z0 = zn;
            break;
        }
        if (!(zn > lo && zn < hi)) {
            z0 = 0.5 * (lo + hi);  // bisection when the step leaves the bracket
            if (hi - lo <= 1e-15 * z0) break;
            continue;
        }
        z0 = zn;
    }
    double z = z0;
    if (three) {
        // deflation: f = (Z - z0)(Z^2 + p Z + q), p = z0 - 1, q = p z0 + r1
        const double p = z0 - 1.0, q = fma(p, z0, r1);
        const double sd = sqrt(fmax(p * p - 4.0 * q, 0.0));
        const double t = -0.5 * (p + copysign(sd, p));  // stable quadratic roots
        const double q1 = t, q2 = (t != 0.0) ? q / t : t;
        double zl = fmin(z0, fmin(q1, q2)), zv = fmax(z0, fmax(q1, q2));
        bool low = false;
        if (zl > B && zl < zv) {
            // FP32 sign of gbar(zl) - gbar(zv) with its error bound (above)
            const float ABf = (float)(A / B);
            const float t1 = (float)(zl - zv), t2 = logf((float)(zl - B)), t3 = logf((float)(zv - B));
            const float t4 = ABf * log1pf((float)(B / zl)), t5 = ABf * log1pf((float)(B / zv));
            const float dg = t1 - (t2 - t3) - (t4 - t5);
            const float tau = 1e-5f * (1.0f + fabsf(t1) + fabsf(t2) + fabsf(t3) + fabsf(t4) + fabsf(t5));
            if (fabsf(dg) > tau) {
                low = dg < 0.0f;
            } else {
                zl = cub_polish(zl, r1, r0);
                zv = cub_polish(zv, r1, r0);
                if (zl > B && zl < zv) {
                    const double AB = A / B;
                    const double gl = zl - log_fast(zl - B) - AB * log_fast(1.0 + B / zl);
                    const double gv = zv - log_fast(zv - B) - AB * log_fast(1.0 + B / zv);
                    low = gl < gv;
                }
                z = low ? zl : zv;
                three = false;  // polished already
            }
        }
        if (three) z = cub_polish(low ? zl : zv, r1, r0);
    }
    Root r;
    r.Z = z;
    r.lzb = log_fast(z - B);
    r.L = log_fast(1.0 + B / z);
    return r;
}

// ---------------------------------------------------------------------------
// Phase evaluation: mixing rules (Eq. mixing_rule), root, ln phi (Eq. lnphi):
// ln phi_i = B_i [(Z - 1)/B + A L / B^2] - ln(Z - B) - psi_i (2 L / B),
// psi_i = sqrt(A_i) sum_j (1 - k_ij) sqrt(A_j) c_j.
// ---------------------------------------------------------------------------
// ln phi_i = B_i u - ln(Z - B) - psi_i v with u = [(Z - 1) + A L / B] / B and
// v = 2 L / B: the scalar coefficients, then one row (shared by the one-lane
// and the several-lanes-per-run evaluations, so both round alike)
__device__ __forceinline__ void lnphi_coef(double A, double B, const Root& r, double& u, double& v) {
    const double invB = 1.0 / B;
    u = ((r.Z - 1.0) + A * r.L * invB) * invB;
    v = 2.0 * r.L * invB;
}
__device__ __forceinline__ double lnphi_row(double Bi, double psi, double u, double v, double lzb) {
    return fma(Bi, u, -lzb) - psi * v;
}

template <int NC>
struct Phase {
    double A, B, Z, L;
    double psi[NC];
    double lnphi[NC];
};

template <int NC>
__device__ __forceinline__ void eos(const Comp<NC>& cp, const Mix<NC>& mx, const double* c, Phase<NC>& ph) {
    double sc[NC];
#pragma unroll
    for (int j = 0; j < NC; j++) sc[j] = mx.sA[j] * c[j];
    double A = 0.0, B = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        double acc = sc[i];  // k_ii = 0
#pragma unroll
        for (int j = 0; j < NC; j++)
            if (j != i) acc = fma(cp.kk[i * NC + j], sc[j], acc);
        ph.psi[i] = mx.sA[i] * acc;
        A = fma(c[i], ph.psi[i], A);
        B = fma(c[i], mx.B[i], B);
    }
    Root r = cubic_select(A, B);
    double u, v;
    lnphi_coef(A, B, r, u, v);
#pragma unroll
    for (int i = 0; i < NC; i++) ph.lnphi[i] = lnphi_row(mx.B[i], ph.psi[i], u, v, r.lzb);
    ph.A = A;
    ph.B = B;
    ph.Z = r.Z;
    ph.L = r.L;
}

// ---------------------------------------------------------------------------
// J_ij = n_T d ln phi_i / d n_j (Appendix A, last paragraph), lower triangle
// of the symmetric matrix, packed row-wise: J[i (i+1)/2 + j], j <= i.
// Differentiating Eq. lnphi through A(c), B(c), psi(c) and the implicit Z of
// the cubic with c_k independent gives f_ik; J_ij = f_ij - sum_k c_k f_ik,
// where the row sums reduce to closed forms (e_i is homogeneous of degree 0).
// ---------------------------------------------------------------------------
//
// R is the type of the per-component vectors and of J.  R = float gives the
// trust regions' model (the Hessians only shape the steps; every point the
// steps reach is evaluated, and every decision taken, in FP64): the scalar
// prelude, where Z - B and the derivative of the cubic can cancel, stays FP64.
// The scalar prelude, the per-component vectors and one entry, shared by the
// one-lane and the several-lanes-per-run evaluations.  Every product and sum
// is explicit (round-to-nearest intrinsics, which are never fused, or fma),
// so the compiler cannot contract them differently in the two contexts and
// both give the same bits.
template <class R>
__device__ __forceinline__ R mul_rn(R a, R b) {
    if constexpr (sizeof(R) == sizeof(float)) return __fmul_rn(a, b);
    else return __dmul_rn(a, b);
}
template <class R>
__device__ __forceinline__ R add_rn(R a, R b) {
    if constexpr (sizeof(R) == sizeof(float)) return __fadd_rn(a, b);
    else return __dadd_rn(a, b);
}
template <class R>
__device__ __forceinline__ R sub_rn(R a, R b) {
    if constexpr (sizeof(R) == sizeof(float)) return __fsub_rn(a, b);
    else return __dsub_rn(a, b);
}

template <class R>
struct DlnPre {
    R fa2, fb, izpb, iz, ib, izb, a, zm1, cl, zcm, lc, qcr;
};

template <class R>
__device__ __forceinline__ DlnPre<R> dln_prelude(double A, double B, double Z, double L) {
    const double FZ = fma(fma(3.0, Z, -2.0), Z, fma(-B, B, sub_rn(A, B)));  // f'(Z)
    const double FA = sub_rn(Z, B), FB = sub_rn(fma(-2.0 * B, Z, -Z), A);
    // the five reciprocals 1/B, 1/(Z-B), 1/(Z+B), 1/Z, 1/FZ from one division
    // (each product of the others and the reciprocal of the whole product)
    const double ZpB = add_rn(Z, B);
    const double p1 = mul_rn(B, FA), p2 = mul_rn(p1, ZpB), p3 = mul_rn(p2, Z);
    const double r4 = 1.0 / mul_rn(p3, FZ);
    const double invFZ = mul_rn(r4, p3), r3 = mul_rn(r4, FZ);
    const double invZ = mul_rn(r3, p2), r2 = mul_rn(r3, Z);
    const double invZpB = mul_rn(r2, p1), r1 = mul_rn(r2, ZpB);
    const double invZB = mul_rn(r1, B), invB = mul_rn(r1, FA);
    const double cL = mul_rn(2.0 * L, invB);  // 2 L / B
    const double Zm1 = sub_rn(Z, 1.0);
    // Zc = sum c_k Z_k, Lc = sum c_k L_k
    const double Zc = mul_rn(-fma(FA, 2.0 * A, mul_rn(FB, B)), invFZ);
    const double Lc = fma(add_rn(Zc, B), invZpB, -mul_rn(Zc, invZ));
    const double qc = mul_rn(sub_rn(Zc, B), invZB);
    DlnPre<R> c;
    c.fa2 = (R)mul_rn(2.0 * FA, invFZ);
    c.fb = (R)mul_rn(FB, invFZ);
    c.izpb = (R)invZpB;
    c.iz = (R)invZ;
    c.ib = (R)invB;
    c.izb = (R)invZB;
    c.a = (R)A;
    c.zm1 = (R)Zm1;
    c.cl = (R)cL;
    c.zcm = (R)sub_rn(Zc, Zm1);
    c.lc = (R)Lc;
    c.qcr = (R)qc;
    return c;
}

// f_ij = bb_i p_j + q_j + psi_i w_j + e_i L_j - cL Ahat_ij with
//   p_j = Z_j - bb_j (Z - 1) + cL (psi_j - A bb_j), q_j = -(Z_j - B_j)/(Z - B),
//   w_j = cL bb_j; the row sum of c_k f_ik is s_i (closed form).
template <class R>
struct DlnVec {
    R bb, p, q, w, e, Lk, sAc, si;
};

template <class R>
__device__ __forceinline__ DlnVec<R> dln_vec(const DlnPre<R>& c, R Bk, R psik, R sAk) {
    DlnVec<R> v;
    const R Zk = -fma(c.fa2, psik, mul_rn<R>(c.fb, Bk));
    v.Lk = fma(add_rn<R>(Zk, Bk), c.izpb, -mul_rn<R>(Zk, c.iz));
    v.bb = mul_rn<R>(Bk, c.ib);
    const R abb = mul_rn<R>(c.a, v.bb);
    v.e = mul_rn<R>(sub_rn<R>(abb, R(2) * psik), c.ib);
    v.p = fma(c.cl, sub_rn<R>(psik, abb), fma(-v.bb, c.zm1, Zk));
    v.q = mul_rn<R>(sub_rn<R>(Bk, Zk), c.izb);
    v.w = mul_rn<R>(c.cl, v.bb);
    v.sAc = mul_rn<R>(c.cl, sAk);
    v.si = fma(v.e, c.lc, fma(v.bb, c.zcm, -c.qcr));
    return v;
}

// entry (i, j), j <= i: row quantities of i, column quantities of j, and
// cL Ahat_ij = ah1 ah2.  Every operation is explicit (fma, or a subtraction
// of two values that are no products), so the compiler cannot contract it
// differently where i == j is known at compile time and where it is not.
template <class R>
__device__ __forceinline__ R dln_entry(R bbi, R psii, R ei, R sii, R pj, R wj, R Lj, R qj, R ah1, R ah2) {
    return fma(bbi, pj, fma(psii, wj, fma(ei, Lj, fma(-ah1, ah2, qj - sii))));
}

template <int NC, class R>
__device__ __forceinline__ void dlnphi_dn_r(const Comp<NC>& cp, const Mix<NC>& mx, const Phase<NC>& ph, R* J) {
    const DlnPre<R> c = dln_prelude<R>(ph.A, ph.B, ph.Z, ph.L);
    DlnVec<R> v[NC];
    R sA[NC], psi[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) {
        psi[k] = (R)ph.psi[k];
        sA[k] = (R)mx.sA[k];
        v[k] = dln_vec<R>(c, (R)mx.B[k], psi[k], sA[k]);
    }
#pragma unroll
    for (int i = 0; i < NC; i++) {
#pragma unroll
        for (int j = 0; j <= i; j++) {
            R kk;
            if constexpr (sizeof(R) == sizeof(float)) kk = cp.kkf[i * NC + j];
            else kk = cp.kk[i * NC + j];
            const R ah1 = (i == j) ? v[i].sAc : mul_rn<R>(kk, v[i].sAc);  // cL Ahat_ij = ah1 sA_j
            J[i * (i + 1) / 2 + j] =
                dln_entry<R>(v[i].bb, psi[i], v[i].e, v[i].si, v[j].p, v[j].w, v[j].Lk, v[j].q, ah1, sA[j]);
        }
    }
}

template <int NC>
__device__ __forceinline__ void dlnphi_dn(const Comp<NC>& cp, const Mix<NC>& mx, const double* c, const Phase<NC>& ph,
                                          double* J) {
    dlnphi_dn_r<NC, double>(cp, mx, ph, J);
}

// ---------------------------------------------------------------------------
// FP32 copy of the phase evaluation (Eqs. mixing_rule, cubic_Z, lnphi), used
// only by the FP32 pre-iteration of stability analysis, whose iterates the
// FP64 iteration then finishes: every decision and every reported number
// comes from FP64.  Same steps as eos and cubic_select (bracketed Halley, root
// count from the critical points, deflation, lower gbar), FP32 arithmetic and
// intrinsics; ln(1 + B/Z) by log1pf (B/Z can be 1e-4).  Returns false on a
// non-finite result.
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ bool eos_f(const Comp<NC>& cp, const float* sA, const float* Bi, const float* c,
                                     float* lnphi) {
    float sc[NC], psi[NC], A = 0.0f, B = 0.0f;
#pragma unroll
    for (int j = 0; j < NC; j++) sc[j] = sA[j] * c[j];
#pragma unroll
    for (int i = 0; i < NC; i++) {
        float acc = sc[i];
#pragma unroll
        for (int j = 0; j < NC; j++)
            if (j != i) acc = fmaf(cp.kkf[i * NC + j], sc[j], acc);
        psi[i] = sA[i] * acc;
        A = fmaf(c[i], psi[i], A);
        B = fmaf(c[i], Bi[i], B);
    }
    const float r1 = A - B * (1.0f + B), r0 = A * B;
    float lo = B, hi = 1.0f + B, z = hi;
#pragma unroll 1
    for (int it = 0; it < 40; it++) {
        const float f = fmaf(fmaf(z - 1.0f, z, r1), z, -r0);
        if (f < 0.0f) lo = z; else hi = z;
        const float fp = fmaf(fmaf(3.0f, z, -2.0f), z, r1), fpp = fmaf(6.0f, z, -2.0f);
        float zn = z - __fdividef(2.0f * f * fp, 2.0f * fp * fp - f * fpp);
        if (fabsf(zn - z) <= 1e-6f * z) {
            z = zn;
            break;
        }
        if (!(zn > lo && zn < hi)) zn = 0.5f * (lo + hi);
        z = zn;
    }
    float Z = z;
    const float dc = fmaf(-12.0f, r1, 4.0f);
    if (dc > 0.0f) {
        const float sq = sqrtf(dc);
        const float zm = (2.0f - sq) * (1.0f / 6.0f), zp = (2.0f + sq) * (1.0f / 6.0f);
        const float fm = fmaf(fmaf(zm - 1.0f, zm, r1), zm, -r0), fpv = fmaf(fmaf(zp - 1.0f, zp, r1), zp, -r0);
        if (!(fm < 0.0f) && !(fpv > 0.0f)) {
            const float p = z - 1.0f, q = fmaf(p, z, r1);
            const float sd = sqrtf(fmaxf(p * p - 4.0f * q, 0.0f));
            const float t = -0.5f * (p + copysignf(sd, p));
            const float q1 = t, q2 = (t != 0.0f) ? q / t : t;
            const float zl = fminf(z, fminf(q1, q2)), zv = fmaxf(z, fmaxf(q1, q2));
            if (zl > B && zl < zv) {
                const float AB = A / B;
                const float gl = zl - __logf(zl - B) - AB * log1pf(B / zl);
                const float gv = zv - __logf(zv - B) - AB * log1pf(B / zv);
                Z = gl < gv ? zl : zv;
            }
        }
    }
    const float lzb = __logf(Z - B), L = log1pf(B / Z);
    const float invB = 1.0f / B;
    const float u = ((Z - 1.0f) + A * L * invB) * invB, v = 2.0f * L * invB;
    bool ok = isfinite(u) && isfinite(v) && isfinite(lzb);
#pragma unroll
    for (int i = 0; i < NC; i++) lnphi[i] = fmaf(Bi[i], u, -lzb) - psi[i] * v;
    return ok;
}

// ---------------------------------------------------------------------------
// Rachford-Rice (Eq. RR) on the Leibovici-Neoschil window (Appendix C):
// Newton on h = (theta - a_l)(a_r - theta) f_RR inside a shrinking bracket,
// bisection when Newton leaves it; stops after a Newton step below 1e-8
// (quadratic convergence leaves an error of order 1e-16).  Returns false if
// K does not bracket 1.  On success t[i] = 1 / (1 + (K_i - 1) theta).
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ bool rachford_rice(const double* z, const double* K, double& theta, double* t) {
    double kmax = K[0], kmin = K[0];
#pragma unroll
    for (int i = 1; i < NC; i++) {
        kmax = fmax(kmax, K[i]);
        kmin = fmin(kmin, K[i]);
    }
    if (!(kmax > 1.0 && kmin < 1.0)) return false;
    const double al = 1.0 / (1.0 - kmax), ar = 1.0 / (1.0 - kmin);
    double lo = al, hi = ar;
    double th = theta;
    if (!(th > lo && th < hi)) th = 0.5 * (fmax(lo, 0.0) + fmin(hi, 1.0));
    double km1[NC];
#pragma unroll
    for (int i = 0; i < NC; i++) km1[i] = K[i] - 1.0;
    {
        // FP32 run of the same iteration from the same start: it seeds the
        // FP64 run, which then needs about two steps (FP32 operations cost a
        // small fraction of an FP64 one here)
        const float alf = (float)al, arf = (float)ar;
        float lof = alf, hif = arf, tf = (float)th;
        float k1f[NC], zf[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) {
            k1f[i] = (float)km1[i];
            zf[i] = (float)z[i];
        }
#pragma unroll 1
        for (int it = 0; it < 60; it++) {
            float f = 0.0f, fp = 0.0f;
#pragma unroll
            for (int i = 0; i < NC; i++) {
                const float a = __fdividef(k1f[i], fmaf(k1f[i], tf, 1.0f));
                f = fmaf(a, zf[i], f);
                fp = fmaf(-a * a, zf[i], fp);
            }
            if (f > 0.0f) lof = tf; else hif = tf;
            const float g1 = tf - alf, g2 = arf - tf;
            const float tn = tf - (g1 * g2 * f) / ((g2 - g1) * f + g1 * g2 * fp);
            if (fabsf(tn - tf) <= 1e-6f * fmaxf(1.0f, fabsf(tf))) {
                tf = tn;
                break;
            }
            tf = (tn > lof && tn < hif) ? tn : 0.5f * (lof + hif);
            if (!(lof < hif)) break;
        }
        const double ts = (double)tf;
        if (ts > lo && ts < hi) th = ts;
    }
#pragma unroll 1
    for (int it = 0; it < 200; it++) {
        double f = 0.0, fp = 0.0;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            double ti = 1.0 / fma(km1[i], th, 1.0);
            double a = km1[i] * ti;
            f = fma(a, z[i], f);
            fp = fma(-a * a, z[i], fp);
        }
        if (f > 0.0) lo = th; else hi = th;
        double g1 = th - al, g2 = ar - th;
        double h = g1 * g2 * f;
        double hp = (g2 - g1) * f + g1 * g2 * fp;
        double tn = th - h / hp;
        // stop once the Newton step is below 1e-8 (Appendix C); the step just
        // taken leaves an error of order its square
        if (fabs(tn - th) <= 1e-8 * fmax(1.0, fabs(th))) {
            th = tn;
            break;
        }
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);  // bisection
        th = tn;
        if (lo >= hi) break;
    }
#pragma unroll
    for (int i = 0; i < NC; i++) t[i] = 1.0 / fma(km1[i], th, 1.0);
    theta = th;
    return true;
}

// FP32 Rachford-Rice for the FP32 precheck evaluations: the same iteration
// as rachford_rice in FP32 (stop at a step below 1e-6 relative).
template <int NC>
__device__ __forceinline__ bool rachford_rice_f(const float* z, const float* K, float& theta, float* t) {
    float kmax = K[0], kmin = K[0];
#pragma unroll
    for (int i = 1; i < NC; i++) {
        kmax = fmaxf(kmax, K[i]);
        kmin = fminf(kmin, K[i]);
    }
    if (!(kmax > 1.0f && kmin < 1.0f)) return false;
    const float al = 1.0f / (1.0f - kmax), ar = 1.0f / (1.0f - kmin);
    float lo = al, hi = ar, th = theta;
    if (!(th > lo && th < hi)) th = 0.5f * (fmaxf(lo, 0.0f) + fminf(hi, 1.0f));
    float km1[NC];
#pragma unroll
    for (int i = 0; i < NC; i++) km1[i] = K[i] - 1.0f;
#pragma unroll 1
    for (int it = 0; it < 60; it++) {
        float f = 0.0f, fp = 0.0f;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            const float a = __fdividef(km1[i], fmaf(km1[i], th, 1.0f));
            f = fmaf(a, z[i], f);
            fp = fmaf(-a * a, z[i], fp);
        }
        if (f > 0.0f) lo = th; else hi = th;
        const float g1 = th - al, g2 = ar - th;
        float tn = th - (g1 * g2 * f) / ((g2 - g1) * f + g1 * g2 * fp);
        if (fabsf(tn - th) <= 1e-6f * fmaxf(1.0f, fabsf(th))) {
            th = tn;
            break;
        }
        th = (tn > lo && tn < hi) ? tn : 0.5f * (lo + hi);
        if (!(lo < hi)) break;
    }
#pragma unroll
    for (int i = 0; i < NC; i++) t[i] = 1.0f / fmaf(km1[i], th, 1.0f);
    theta = th;
    return true;
}

// ---------------------------------------------------------------------------
// Small dense linear algebra on packed lower triangles (n <= 16), per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// The routines below take the matrix in FP64 (H, packed lower triangle) and
// work in R: R = float for the trust regions' model steps (factorisation,
// triangular solves, the shift iteration), R = double where a Newton step must
// be exact to FP64 (the split's polish once an FP32-model step fell short).
template <class R>
__device__ __forceinline__ R rsqrt_r(R d) {
    if constexpr (sizeof(R) == sizeof(float)) return rsqrtf(d);
    else return rsqrt(d);
}

// Cholesky of (H + eta diag(1)) in the scaled space; returns -1 if positive
// definite, else the column j whose pivot d_j <= 0 (in *dfail).  Lf holds L
// below the diagonal and 1 / L_jj on it, so that the triangular solves
// multiply instead of divide (FP64 division costs ~7 FMA slots here).
template <int NC, class R>
__device__ __forceinline__ int cholesky(const double* H, R eta, R* Lf, R* dfail) {
#pragma unroll 1
    for (int j = 0; j < NC; j++) {
        R d = (R)H[tri(j, j)] + eta;
#pragma unroll 1
        for (int k = 0; k < j; k++) d = fma(-Lf[tri(j, k)], Lf[tri(j, k)], d);
        if (!(d > R(0))) {
            *dfail = d;
            return j;
        }
        const R inv = rsqrt_r(d);
        Lf[tri(j, j)] = inv;
#pragma unroll 1
        for (int i = j + 1; i < NC; i++) {
            R s = (R)H[tri(i, j)];
#pragma unroll 1
            for (int k = 0; k < j; k++) s = fma(-Lf[tri(i, k)], Lf[tri(j, k)], s);
            Lf[tri(i, j)] = s * inv;
        }
    }
    return -1;
}

// After a factorisation of H + eta I failed at column j with pivot d <= 0:
// w = (-L1^{-T} l, 1, 0, ...), with L1 the leading j x j factor and l the
// computed part of row j, has w.(H + eta I).w = d, so the smallest eigenvalue
// of H is at most d / ||w||^2 - eta (More and Sorensen 1983, Sec. 3).
// Returns that bound on -lambda_min: eta - d / ||w||^2.
template <int NC, class R>
__device__ __forceinline__ double shift_bound(const R* Lf, int j, R d, double eta) {
    R w[NC], wn = R(1);
#pragma unroll 1
    for (int i = j - 1; i >= 0; i--) {
        R s = -Lf[tri(j, i)];
#pragma unroll 1
        for (int k = i + 1; k < j; k++) s = fma(-Lf[tri(k, i)], w[k], s);
        w[i] = s * Lf[tri(i, i)];
        wn = fma(w[i], w[i], wn);
    }
    return eta - (double)d / (double)wn;
}

// Solve L y = b (forward) in place
template <int NC, class R>
__device__ __forceinline__ void fwd(const R* Lf, R* b) {
#pragma unroll 1
    for (int i = 0; i < NC; i++) {
        R s = b[i];
#pragma unroll 1
        for (int k = 0; k < i; k++) s = fma(-Lf[tri(i, k)], b[k], s);
        b[i] = s * Lf[tri(i, i)];
    }
}

// Solve L^T x = b (backward) in place
template <int NC, class R>
__device__ __forceinline__ void bwd(const R* Lf, R* b) {
#pragma unroll 1
    for (int i = NC - 1; i >= 0; i--) {
        R s = b[i];
#pragma unroll 1
        for (int k = i + 1; k < NC; k++) s = fma(-Lf[tri(k, i)], b[k], s);
        b[i] = s * Lf[tri(i, i)];
    }
}

// Trust-region subproblem (Appendix B): minimise gs.u + u.Hs.u/2 subject to
// ||u|| <= radius in the scaled space, by Hebden's iteration on the shift eta
// of (Hs + eta I) u = -gs (Hebden 1973; More and Sorensen 1983), solved to
// kShiftTol = 1e-4 relative on ||u||: the radius is a safeguard on the step,
// so a step within 1e-4 of it serves the ratio test and the radius update as
// well as the exact one (at 1e-10 the longest runs took 3.4 factorisations
// per trip).
//
// One call does one factorisation, so a persistent kernel spends one
// factorisation per lane per trip and a lane that needs many shifts does not
// hold its warp-mates inside a loop:
//  - a fresh solve factors at eta = 0 and takes the Newton step when H is
//    positive definite and the step fits;
//  - otherwise it brackets the shift [elo, ehi] (Gershgorin and ||g|| / radius)
//    and each further call takes one Newton step on 1/||u(eta)|| - 1/radius.
//    A failed factorisation raises elo to its pivot's eigenvalue bound; a
//    failure or a step that leaves the bracket continues from the safeguarded
//    geometric midpoint max(sqrt(elo ehi), elo + 1e-3 (ehi - elo)) (More and
//    Sorensen 1983, Sec. 3).  After kTRShiftCap calls the next positive
//    definite factorisation ends the solve, so a solve takes at most
//    kTRShiftCap + 2 calls.
//    From the left of the solution these steps never overshoot (the function
//    is concave), so the first starts from the eta = 0 factorisation, and a
//    caller that shrank the radius around the same H passes the previous shift
//    as a further lower bound.
//  - warm start (More and Sorensen 1983, Sec. 4): a run whose previous solve
//    ended on the boundary (sh.warm > 0, that solve's shift) starts the next
//    one from that shift, inside the new bracket, instead of from eta = 0:
//    the shift changes little from trip to trip.  If the step there falls
//    short of the radius and nothing excludes eta = 0 (elo == 0), eta = 0 is
//    tried next, where a Newton step that fits ends the solve.
//  - the iteration also stops once the bracket has closed to 1e-12 relative
//    (1e-6 in FP32): with the shift at the pole -lambda_min (the nearly hard
//    case) ||u|| can change by 1e-8 relative for the smallest change of eta.
// A radius <= 0 is not yet set: it becomes ||Newton step|| when H is positive
// definite, else 1.  Returns 1 with the step in u (the shift used in sh.eta),
// 0 if the iteration continues on the next call, and -1 with newton_only when
// H is not positive definite, or when the solve failed: a factorisation that
// fails even at the upper end of the bracket (a matrix that is not finite in
// R) would otherwise repeat forever, so past kTRShiftCap + 2 calls the solve
// gives up (the solve is then over: sh.active = 0).
constexpr int kTRShiftCap = 40;

struct TRShift {
    double eta, elo, ehi;
    double warm;  // shift of the run's last boundary step (0: none yet, or an interior step)
    int active, it;
    int zero;     // this solve has factored at eta = 0
};

// The shift bracket of a fresh solve: Gershgorin bounds of H and ||g|| / radius
template <int NC>
__device__ __forceinline__ void shift_bracket(const double* Hs, const double* gs, double radius, double eta_lo,
                                              TRShift& sh) {
    double gn = 0.0, hn1 = 0.0, mind = 1e300;
#pragma unroll 1
    for (int i = 0; i < NC; i++) {
        gn = fma(gs[i], gs[i], gn);
        double rs = 0.0;
#pragma unroll 1
        for (int j = 0; j < NC; j++) rs += fabs(Hs[i >= j ? tri(i, j) : tri(j, i)]);
        hn1 = fmax(hn1, rs);
        mind = fmin(mind, Hs[tri(i, i)]);
    }
    gn = sqrt(gn);
    sh.elo = fmax(fmax(0.0, eta_lo), fmax(-mind, gn / radius - hn1));
    sh.ehi = gn / radius + hn1;
    sh.active = 1;
    sh.it = 0;
}

template <int NC, class R>
__device__ __forceinline__ int tr_shift_step(const double* Hs, const double* gs, double& radius, double eta_lo,
                                             bool newton_only, TRShift& sh, R* Lf, double* u) {
    constexpr double kShiftTol = 1e-4;
    constexpr double kPoleTol = sizeof(R) == sizeof(float) ? 1e-6 : 1e-12;
    if (sh.active && sh.it > kTRShiftCap + 2) {
        sh.active = 0;
        return -1;
    }
    if (!sh.active && !newton_only && sh.warm > 0.0 && radius > 0.0) {
        shift_bracket<NC>(Hs, gs, radius, eta_lo, sh);
        sh.zero = 0;
        sh.eta = fmin(fmax(sh.warm, sh.elo), sh.ehi);
    }
    const double eta = sh.active ? sh.eta : 0.0;
    R dfail = R(0);
    const int jf = cholesky<NC, R>(Hs, (R)eta, Lf, &dfail);
    const bool pd = jf < 0;
    double un = 0.0;
    R ur[NC];
    if (pd) {
#pragma unroll
        for (int i = 0; i < NC; i++) ur[i] = (R)(-gs[i]);
        fwd<NC, R>(Lf, ur);
        bwd<NC, R>(Lf, ur);
#pragma unroll
        for (int i = 0; i < NC; i++) u[i] = (double)ur[i];
        if (newton_only) return 1;
#pragma unroll
        for (int i = 0; i < NC; i++) un = fma(u[i], u[i], un);
        un = sqrt(un);
        if (!sh.active) {
            if (radius <= 0.0) radius = un;
            if (un <= radius) {
                sh.eta = 0.0;
                sh.warm = 0.0;
                return 1;
            }
        } else if (eta == 0.0 && un <= radius) {  // a warm start back at eta = 0: the Newton step fits
            sh.active = 0;
            sh.eta = 0.0;
            sh.warm = 0.0;
            return 1;
        } else if (fabs(un - radius) <= kShiftTol * radius || sh.it >= kTRShiftCap) {
            sh.active = 0;
            sh.warm = eta;
            return 1;
        }
    } else if (newton_only) {
        return -1;
    }
    if (!sh.active) {
        if (radius <= 0.0) radius = 1.0;
        shift_bracket<NC>(Hs, gs, radius, eta_lo, sh);
        sh.zero = 1;
    }
    sh.it++;
    if (!pd) {
        // eigenvalue bound from the failed pivot, then the safeguarded
        // midpoint of the bracket; past the cap the upper end, where H + eta I
        // is positive definite, so that the next call ends the solve
        sh.elo = fmax(sh.elo, shift_bound<NC, R>(Lf, jf, dfail, eta));
        if (!(sh.ehi > sh.elo)) sh.ehi = 2.0 * sh.elo + 1e-300;
        sh.eta = sh.it >= kTRShiftCap ? sh.ehi
                                      : fmax(sqrt(fmax(sh.elo, 1e-300) * sh.ehi), sh.elo + 1e-3 * (sh.ehi - sh.elo));
        return 0;
    }
    if (!(sh.ehi > sh.elo)) sh.ehi = 2.0 * sh.elo + 1e-300;
    // positive definite, ||u|| off the radius: Newton step on the secular equation
    if (un < radius) sh.ehi = eta;
    else sh.elo = fmax(sh.elo, eta);
    if (un < radius && !sh.zero && sh.elo == 0.0) {  // warm start right of the root: eta = 0 first
        sh.zero = 1;
        sh.eta = 0.0;
        return 0;
    }
    if (sh.ehi - sh.elo <= kPoleTol * sh.ehi) {  // shift pinned at the pole: ||u|| is as close as it gets
        sh.active = 0;
        sh.eta = eta;
        sh.warm = eta;
        return 1;
    }
    R q[NC];
    double qn = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) q[i] = ur[i];
    fwd<NC, R>(Lf, q);
#pragma unroll
    for (int i = 0; i < NC; i++) qn = fma((double)q[i], (double)q[i], qn);
    double en = eta + (un * un / qn) * (un - radius) / radius;
    if (un > radius) en = fmax(en, sh.elo);
    if (!(en >= sh.elo && en < sh.ehi)) {  // out of the bracket: geometric midpoint
        en = fmax(sqrt(fmax(sh.elo, 1e-300) * sh.ehi), sh.elo + 1e-3 * (sh.ehi - sh.elo));
    }
    if (en == eta) {  // no representable progress: take this step
        sh.active = 0;
        sh.eta = eta;
        sh.warm = eta;
        return 1;
    }
    sh.eta = en;
    return 0;
}

// DEM factor (Sec. 2.2.1, reading R7): lambda = (dk.d1)/(d1.d1), used when
// the updates shrink and 0 < lambda < 1; returns lambda / (1 - lambda) or 0.
// Applied on every kDemPeriod-th update of an SS run.
constexpr int kDemPeriod = 3;

template <int NC>
__device__ __forceinline__ double dem_factor(const double* dk, const double* d1) {
    double n0 = 0.0, n1 = 0.0, p01 = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        n0 = fma(dk[i], dk[i], n0);
        n1 = fma(d1[i], d1[i], n1);
        p01 = fma(dk[i], d1[i], p01);
    }
    if (!(n1 > 0.0) || !(n0 < n1)) return 0.0;
    const double lam = p01 / n1;
    if (!(lam > 0.0 && lam < 1.0)) return 0.0;
    return lam / (1.0 - lam);
}

// FP32 copy for the FP32 stability pre-iteration
template <int NC>
__device__ __forceinline__ float dem_factor_f(const float* dk, const float* d1) {
    float n0 = 0.0f, n1 = 0.0f, p01 = 0.0f;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        n0 = fmaf(dk[i], dk[i], n0);
        n1 = fmaf(d1[i], d1[i], n1);
        p01 = fmaf(dk[i], d1[i], p01);
    }
    if (!(n1 > 0.0f) || !(n0 < n1)) return 0.0f;
    const float lam = p01 / n1;
    if (!(lam > 0.0f && lam < 1.0f)) return 0.0f;
    return lam / (1.0f - lam);
}

template <int NC>
__device__ __forceinline__ double maxabs(const double* v) {
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) r = fmax(r, fabs(v[i]));
#pragma unroll
    for (int i = 0; i < NC; i++)
        if (v[i] != v[i]) r = INFINITY;
    return r;
}

}  // namespace ptf
