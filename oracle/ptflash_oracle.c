/*
 * ptflash_oracle.c -- CPU oracle for the batched isothermal two-phase flash
 * (arXiv 2205.03090, "PTFlash").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, FP64 restatement of
 * the method that the CUDA path is checked against.  Only tests/, the smoke
 * check and the CPU-baseline leg of bench.py may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Every function cites the section / equation of the paper it follows.  Where
 * the paper is silent or garbled, the reading taken is written next to the
 * code and listed in the design notes:
 *   R1  R cancels from A_i and B_i (Appendix A, Eq. a_i, b_i, A, B).
 *   R2  Michelsen's tm: tm = 1 + sum W_i (ln W_i + ln phi_i(W) - d_i - 1)
 *       (Sec. 2.2.1, Eq. tm printed without the leading 1).
 *   R3  Delta G = theta tpd(y) + (1 - theta) tpd(x) (Sec. 2.2.3; the printed
 *       weights pair theta with the vapour trial).
 *   R4  Stability Hessian uses d ln phi_i / d W_j (Appendix B, Eq. analysis_hess
 *       index typo).
 *   R5  Split Hessian uses the unit-total-mole derivatives
 *       n_T d ln phi / d n, weighted theta for the liquid and 1-theta for the
 *       vapour (Appendix B, Eq. split_hess).
 *   R6  Root choice: among real roots Z > B, the smallest and the largest
 *       are compared by the residual Gibbs energy
 *       gbar(Z) = Z - 1 - ln(Z - B) - (A/B) ln(1 + B/Z); the lower wins
 *       (Appendix A, after Eq. halley).
 *   R7  DEM: lambda = (D_k . D_{k-1}) / (D_{k-1} . D_{k-1}) on successive
 *       ln K (ln W) updates D; on every 3rd update of a run, if
 *       0 < lambda < 1 and the updates shrink, add D_k lambda / (1 - lambda)
 *       (Sec. 2.2.1 names DEM without its period or safeguards).  If the
 *       next evaluation fails or does not lower the residual the accelerated
 *       update is undone (that evaluation counts toward the iteration cap).
 *       Of the periods and safeguards tried, this one lets the most trials
 *       finish by SS, nearest the SS convergence rates of Table 4.
 *   R8  "Negative" tm / tpd / Delta G means below -EPS_NEG (1e-10).
 *   R9  Trust region: exact subproblem min g.d + d.H.d/2 s.t. ||d||_M <= r;
 *       initial radius = ||Newton step|| if H is positive definite, else 1;
 *       signed ratio rho = actual / predicted; accept iff rho > 0; halve r if
 *       rho <= 0.25, double if rho >= 0.75 (Appendix B).  When the
 *       predicted change is below 1e-12 (1 + |objective|) the ratio is
 *       rounding noise: the step is accepted and the radius kept.  Split
 *       steps keep 0 < n^V_i < z_i by a 0.99 fraction-to-boundary cut.
 *   R10 Split convergence tightened from the printed 1e-8 to the fugacity
 *       residual 1e-10; trust-region runs stop at the printed 1e-8 and then
 *       take plain Newton steps until the residual is <= 1e-10 (at least one,
 *       at most 10).  The paper caps the stability trust region at 20
 *       iterations (Alg. 2) but gives no cap for the split one (its Table 4
 *       run needed at most 13): a cap of 60 lets the slow split runs near
 *       three-phase conditions converge (the slowest seen took 33 iterations
 *       with the polish), where a cap of 20 left 13 of 2e5 8-component
 *       mixtures unconverged.
 *   R11 Precheck: 3 SS evaluations from Wilson K; theta outside (0,1) or no
 *       Rachford-Rice root at any of them routes to stability; otherwise the
 *       tests use x, y of the 3rd evaluation and the split continues from
 *       the 3rd update with a fresh cap of 9 (Sec. 2.2.3).
 *   R12 Rachford-Rice root sought on the Leibovici-Neoschil window
 *       (1/(1-K_max), 1/(1-K_min)); theta outside (0,1) is allowed inside
 *       the split iterations (negative flash).
 *   R13 A split whose K collapse to 1 (max |ln K| < 1e-6), or that converges
 *       with theta outside (0,1), or whose K stop bracketing 1, is reported
 *       single-phase with the COLLAPSE status bit.  An SS run that reaches
 *       its cap with theta outside (0,1) starts the trust region from the
 *       feasible material-balance point n^V_i = t K_i z_i / (1 + t (K_i - 1))
 *       at t = 1/2.  A trust-region iterate whose theta comes within 1e-10
 *       of 0 or 1 has collapsed onto one phase without converging (each
 *       fraction-to-boundary step then moves theta six decades further): the
 *       run stops there, single-phase with the COLLAPSE and MAXITER bits.
 *   R14 Canonical phase labels: after a two-phase result, if Z(y) < Z(x)
 *       the phases are swapped (y is always the lower-density phase).
 *   R15 Single phase output: beta = 0, x = y = z, K = 1.
 *   R16 K re-estimate from a stability trial (Sec. 2.2.1, last sentence)
 *       uses the trial's composition w = W / sum W: K_i = w_i / z_i for the
 *       vapour-like trial, z_i / w_i for the liquid-like one.  The printed
 *       W^V_i / z_i and z_i / W^L_i agree at a stationary point; after an
 *       early stop at the first negative tm the unnormalised form can give K
 *       that do not bracket 1, and the split then collapses although the
 *       mixture is unstable.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXNC 16

/* status bits (the CUDA library documents the same values) */
#define ST_PRECHECK_UNSTABLE 1
#define ST_STAB_RUN 2
#define ST_STAB_TR 4
#define ST_SPLIT_TR 8
#define ST_MAXITER 16
#define ST_COLLAPSE 32
#define ST_NONFINITE 64

/* constants printed in the paper */
#define SRK_OMEGA_A 0.42748   /* Eq. a_i */
#define SRK_OMEGA_B 0.08664   /* Eq. b_i */
#define WILSON_C 5.373        /* Eq. wilson */
#define TOL_STAB 1e-6         /* Sec. 2.2.1 and Appendix B.1 */
#define TOL_SPLIT_TR 1e-8     /* Appendix B.2 */
#define TOL_FUG 1e-10         /* fugacity residual (R10) */
#define KSS_STAB 9            /* Alg. 2 */
#define KTR_STAB 20           /* Alg. 2 */
#define KSS_SPLIT 9           /* Sec. 2.2.2 */
#define KTR_SPLIT 60          /* R10: the paper gives no split TR cap */
#define KNEWTON_POLISH 10     /* R10 */
#define NPRECHECK 3           /* Sec. 2.2.3 */
#define EPS_NEG 1e-10         /* R8 */
#define TRIVIAL_LNK 1e-6      /* R13 */
#define COLLAPSE_TH 1e-10     /* R13: trust-region iterate collapsed onto one phase */
#define PRED_TRUST 1e-12      /* R9: ratio test trusted above this relative size */

/* ------------------------------------------------------------------------ */
/* Algorithmic FP64 work, counted per stage along the path each mixture      */
/* takes.  Each primitive is charged the operations of the method's own      */
/* numerics (Halley roots, Newton Rachford-Rice, Cholesky trust-region       */
/* steps), not of the oracle's slower bracketing.  Kinds, counted apart:     */
/* plain flops (add, multiply = 1, fused multiply-add = 2), divisions,        */
/* square roots, exponentials, logarithms.  Stages: 0 prep+precheck,         */
/* 1 stability SS, 2 stability TR, 3 split SS, 4 split TR.  This is test     */
/* instrumentation: it does not change what the oracle computes.             */
/* ------------------------------------------------------------------------ */
#define NSTAGE 5
#define NKIND 5 /* flops, divisions, square roots, exponentials, logarithms */
typedef struct { double fl, dv, sq, ex, lg; } or_ops;
static _Thread_local double g_ops[NSTAGE][NKIND];
static _Thread_local int g_stage;
static void count(or_ops o) {
    g_ops[g_stage][0] += o.fl;
    g_ops[g_stage][1] += o.dv;
    g_ops[g_stage][2] += o.sq;
    g_ops[g_stage][3] += o.ex;
    g_ops[g_stage][4] += o.lg;
}
static or_ops ops(double fl, double dv, double sq, double ex, double lg) {
    or_ops o = {fl, dv, sq, ex, lg};
    return o;
}
static or_ops add_ops(or_ops a, or_ops b) { return ops(a.fl + b.fl, a.dv + b.dv, a.sq + b.sq, a.ex + b.ex, a.lg + b.lg); }
static or_ops scale_ops(or_ops a, double k) { return ops(k * a.fl, k * a.dv, k * a.sq, k * a.ex, k * a.lg); }
/* per-primitive counts */
static or_ops cost_eos(int nc, int three) {
    or_ops c = ops(2.0 * nc * nc + 8.0 * nc, 0, 0, 0, 0);   /* mixing sums */
    c = add_ops(c, ops(18.0, 0, 1, 0, 0));                  /* root count: 2 cubic evaluations, sqrt */
    c = add_ops(c, ops(2 * 16.0, 2, 0, 0, 0));              /* two FP64 Halley steps */
    c = add_ops(c, ops(3.0, 1, 0, 0, 2));                   /* ln(Z - B), ln(1 + B/Z) */
    c = add_ops(c, ops(4.0 + 3.0 * nc, 2, 0, 0, 0));        /* ln phi */
    if (three) c = add_ops(c, ops(10.0 + 2 * 8.0 + 8.0, 1 + 2 + 2, 1, 0, 4)); /* deflation, polish, gbar */
    return c;
}
static or_ops cost_jac(int nc) { return ops(7.0 * nc * (nc + 1) + 30.0 * nc, 8, 0, 0, 0); }
static or_ops cost_rr(int nc) { return ops(4.0 * (6.0 * nc + 10.0), 4.0 * (nc + 1) + nc, 0, 0, 0); }
static or_ops cost_chol(int nc) { return ops(2.0 * nc * nc * nc / 6.0 + 2.0 * nc * nc, nc, nc, 0, 0); }
static or_ops cost_trsub(int nc) { return add_ops(scale_ops(cost_chol(nc), 3.0), ops(4.0 * nc * nc, 0, 0, 0, 0)); }

/* ------------------------------------------------------------------------ */
/* Component system and per-mixture EOS constants (Appendix A)              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nc;
    double Tc[OR_MAXNC], Pc[OR_MAXNC], om[OR_MAXNC];
    double kij[OR_MAXNC * OR_MAXNC];
} or_sys;

typedef struct {
    int nc;
    double Ai[OR_MAXNC];  /* a_i alpha_i P / (R T)^2 */
    double Bi[OR_MAXNC];  /* b_i P / (R T) */
    double Aij[OR_MAXNC * OR_MAXNC]; /* (1 - k_ij) sqrt(A_i A_j), Eq. a_ij */
} or_mix;

/* Appendix A, Eqs. a_i, b_i, alpha_i, m_i; A = a alpha P/(R^2 T^2),
 * B = b P/(R T).  With a_i = 0.42748 R^2 Tc^2/Pc the gas constant cancels
 * (reading R1). */
void or_mix_init(const or_sys* s, double P, double T, or_mix* m) {
    m->nc = s->nc;
    for (int i = 0; i < s->nc; i++) {
        double mi = 0.480 + 1.574 * s->om[i] - 0.176 * s->om[i] * s->om[i];
        double a = 1.0 + mi * (1.0 - sqrt(T / s->Tc[i]));
        double alpha = a * a;
        double Tr = T / s->Tc[i], Pr = P / s->Pc[i];
        m->Ai[i] = SRK_OMEGA_A * alpha * Pr / (Tr * Tr);
        m->Bi[i] = SRK_OMEGA_B * Pr / Tr;
    }
    for (int i = 0; i < s->nc; i++)
        for (int j = 0; j < s->nc; j++)
            m->Aij[i * s->nc + j] = (1.0 - s->kij[i * s->nc + j]) * sqrt(m->Ai[i] * m->Ai[j]);
}

/* Eq. wilson */
void or_wilson(const or_sys* s, double P, double T, double* lnK) {
    for (int i = 0; i < s->nc; i++)
        lnK[i] = log(s->Pc[i] / P) + WILSON_C * (1.0 + s->om[i]) * (1.0 - s->Tc[i] / T);
}

/* ------------------------------------------------------------------------ */
/* Cubic in Z (Eq. cubic_Z): all real roots, ascending.                     */
/* f(Z) = Z^3 - Z^2 + rho1 Z - rho0.  The oracle does not use the paper's    */
/* Halley iteration: it brackets every real root between the critical points */
/* of f and bisects (with Newton steps kept inside the bracket) to the last  */
/* representable double, which is path independent.                          */
/* ------------------------------------------------------------------------ */
static double cubic_f(double Z, double r1, double r0) { return ((Z - 1.0) * Z + r1) * Z - r0; }
static double cubic_df(double Z, double r1) { return (3.0 * Z - 2.0) * Z + r1; }

static double bracket_root(double lo, double hi, double r1, double r0) {
    double flo = cubic_f(lo, r1, r0);
    if (flo == 0.0) return lo;
    double fhi = cubic_f(hi, r1, r0);
    if (fhi == 0.0) return hi;
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 400; it++) {
        double fx = cubic_f(x, r1, r0);
        if (fx == 0.0) return x;
        if ((fx < 0.0) == (flo < 0.0)) { lo = x; flo = fx; } else { hi = x; }
        double d = cubic_df(x, r1);
        double xn = (d != 0.0) ? x - fx / d : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (xn == x || hi - lo <= 4.0 * 2.220446049250313e-16 * fabs(x)) {
            x = xn;
            break;
        }
        x = xn;
    }
    return x;
}

int or_cubic_roots(double A, double B, double* roots) {
    double r1 = A - B * (1.0 + B), r0 = A * B;
    double bound = 1.0 + fabs(r1) + fabs(r0) + 1.0; /* all roots in (-bound, bound) */
    double disc = 4.0 - 12.0 * r1;                  /* of f'(Z) = 3Z^2 - 2Z + rho1 */
    if (disc <= 0.0) {
        roots[0] = bracket_root(-bound, bound, r1, r0);
        return 1;
    }
    double sq = sqrt(disc);
    double zm = (2.0 - sq) / 6.0, zp = (2.0 + sq) / 6.0; /* local max, local min */
    double fm = cubic_f(zm, r1, r0), fp = cubic_f(zp, r1, r0);
    int n = 0;
    if (fm < 0.0) {                /* only the root right of the local min */
        roots[n++] = bracket_root(zp, bound, r1, r0);
    } else if (fp > 0.0) {         /* only the root left of the local max */
        roots[n++] = bracket_root(-bound, zm, r1, r0);
    } else {                       /* three real roots (double roots counted twice) */
        roots[n++] = bracket_root(-bound, zm, r1, r0);
        roots[n++] = bracket_root(zm, zp, r1, r0);
        roots[n++] = bracket_root(zp, bound, r1, r0);
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Phase EOS evaluation: mixing rules (Eq. mixing_rule), root selection     */
/* (reading R6) and fugacity coefficients (Eq. lnphi).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double A, B, Z;
    double psi[OR_MAXNC]; /* sum_j A_ij c_j */
    double lnphi[OR_MAXNC];
} or_phase;

static double gbar(double Z, double A, double B) {
    return Z - 1.0 - log(Z - B) - (A / B) * log(1.0 + B / Z);
}

/* Returns 0 on success, -1 if no admissible root. */
int or_eos(const or_mix* m, const double* c, or_phase* ph) {
    int nc = m->nc;
    double A = 0.0, B = 0.0;
    for (int i = 0; i < nc; i++) {
        double p = 0.0;
        for (int j = 0; j < nc; j++) p += m->Aij[i * nc + j] * c[j];
        ph->psi[i] = p;
    }
    for (int i = 0; i < nc; i++) {
        A += c[i] * ph->psi[i];
        B += c[i] * m->Bi[i];
    }
    double r[3];
    int n = or_cubic_roots(A, B, r);
    /* admissible roots are Z > B (positive free volume) */
    double zl = 0.0, zv = 0.0;
    int have = 0;
    for (int k = 0; k < n; k++) {
        if (r[k] > B) {
            if (!have) { zl = r[k]; zv = r[k]; have = 1; }
            else { if (r[k] < zl) zl = r[k]; if (r[k] > zv) zv = r[k]; }
        }
    }
    if (!have) return -1;
    double Z = zv;
    if (zl < zv && gbar(zl, A, B) < gbar(zv, A, B)) Z = zl;
    count(cost_eos(nc, zl < zv));
    ph->A = A;
    ph->B = B;
    ph->Z = Z;
    double L = log(1.0 + B / Z), lzb = log(Z - B);
    for (int i = 0; i < nc; i++) {
        double bb = m->Bi[i] / B;
        ph->lnphi[i] = bb * (Z - 1.0) - lzb + (A / B) * (bb - 2.0 * ph->psi[i] / A) * L;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Derivatives J_ij = n_T d ln phi_i / d n_j at fixed T, P (Appendix A,      */
/* last paragraph: computed explicitly).  Derived by differentiating        */
/* Eq. lnphi through A(c), B(c), psi(c) and the implicit Z(A, B) of the cubic */
/* with c_k treated as independent (f_ik = d ln phi_i / d c_k), then          */
/* J_ij = f_ij - sum_k c_k f_ik  (c = n / n_T).                               */
/* ------------------------------------------------------------------------ */
void or_dlnphi_dn(const or_mix* m, const double* c, const or_phase* ph, double* J) {
    int nc = m->nc;
    count(cost_jac(nc));
    double A = ph->A, B = ph->B, Z = ph->Z;
    double L = log(1.0 + B / Z);
    double FZ = 3.0 * Z * Z - 2.0 * Z + A - B - B * B;
    double FA = Z - B;
    double FB = -Z - 2.0 * B * Z - A;
    double Zk[OR_MAXNC], Lk[OR_MAXNC], e[OR_MAXNC];
    for (int k = 0; k < nc; k++) {
        Zk[k] = -(FA * 2.0 * ph->psi[k] + FB * m->Bi[k]) / FZ;
        Lk[k] = (Zk[k] + m->Bi[k]) / (Z + B) - Zk[k] / Z;
    }
    for (int i = 0; i < nc; i++) e[i] = A * m->Bi[i] / (B * B) - 2.0 * ph->psi[i] / B;
    double f[OR_MAXNC * OR_MAXNC];
    for (int i = 0; i < nc; i++) {
        for (int k = 0; k < nc; k++) {
            double de = 2.0 * ph->psi[k] * m->Bi[i] / (B * B) - 2.0 * A * m->Bi[i] * m->Bi[k] / (B * B * B)
                        - 2.0 * m->Aij[i * nc + k] / B + 2.0 * ph->psi[i] * m->Bi[k] / (B * B);
            f[i * nc + k] = -(m->Bi[i] * m->Bi[k] / (B * B)) * (Z - 1.0) + (m->Bi[i] / B) * Zk[k]
                            - (Zk[k] - m->Bi[k]) / (Z - B) + de * L + e[i] * Lk[k];
        }
    }
    for (int i = 0; i < nc; i++) {
        double s = 0.0;
        for (int k = 0; k < nc; k++) s += c[k] * f[i * nc + k];
        for (int j = 0; j < nc; j++) J[i * nc + j] = f[i * nc + j] - s;
    }
}

/* ------------------------------------------------------------------------ */
/* Rachford-Rice (Eq. RR, Appendix C).  The root of f_RR is unique on the    */
/* Leibovici-Neoschil window (alpha_l, alpha_r), where f_RR decreases        */
/* monotonically.  The oracle bisects f_RR on the window to adjacent doubles */
/* (the paper's Newton/bisection on h_RR reaches the same root).             */
/* Returns 0 and theta, or -1 when K does not bracket 1.                     */
/* ------------------------------------------------------------------------ */
static double rr_f(int nc, const double* z, const double* K, double th) {
    double s = 0.0;
    for (int i = 0; i < nc; i++) s += (K[i] - 1.0) * z[i] / (1.0 + (K[i] - 1.0) * th);
    return s;
}

int or_rr(int nc, const double* z, const double* K, double* theta) {
    double kmax = K[0], kmin = K[0];
    for (int i = 1; i < nc; i++) { if (K[i] > kmax) kmax = K[i]; if (K[i] < kmin) kmin = K[i]; }
    if (!(kmax > 1.0 && kmin < 1.0)) return -1;
    count(cost_rr(nc));
    double lo = 1.0 / (1.0 - kmax), hi = 1.0 / (1.0 - kmin); /* alpha_l < 0 < 1 < alpha_r */
    for (int it = 0; it < 2000; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = rr_f(nc, z, K, mid);
        if (f > 0.0) lo = mid; else if (f < 0.0) hi = mid; else { lo = hi = mid; break; }
    }
    *theta = 0.5 * (lo + hi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra for the trust-region subproblem (Appendix B).  */
/* Symmetric eigendecomposition by cyclic Jacobi rotations.                  */
/* ------------------------------------------------------------------------ */
static void jacobi_eig(int n, const double* Ain, double* lam, double* V) {
    double a[OR_MAXNC * OR_MAXNC];
    memcpy(a, Ain, sizeof(double) * n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                tot += a[i * n + j] * a[i * n + j];
                if (i != j) off += a[i * n + j] * a[i * n + j];
            }
        if (off <= 1e-34 * tot || off == 0.0) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double app = a[p * n + p], aqq = a[q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < n; k++) { /* rotate columns p, q */
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = cs * akp - sn * akq;
                    a[k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; k++) { /* rotate rows p, q */
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = cs * apk - sn * aqk;
                    a[q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = cs * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    for (int i = 0; i < n; i++) lam[i] = a[i * n + i];
}

/* Exact trust-region subproblem in the M-norm (M diagonal, m = diag or NULL
 * for the identity): minimise g.d + d.H.d/2 subject to ||d||_M <= radius.
 * With u = M^{1/2} d the problem is the Euclidean one for
 * H' = M^{-1/2} H M^{-1/2}, g' = M^{-1/2} g.  The multiplier eta >= 0 solves
 * ||u(eta)|| = radius, u(eta) = -(H' + eta I)^{-1} g', found by bisection on
 * the monotone norm; if H' is positive definite and the Newton step fits,
 * eta = 0.  Returns the predicted change g.d + d.H.d/2. */
static double unorm(int n, const double* gt, const double* lam, double eta) {
    double s = 0.0;
    for (int k = 0; k < n; k++) {
        double u = gt[k] / (lam[k] + eta);
        s += u * u;
    }
    return sqrt(s);
}

double or_tr_subproblem(int n, const double* H, const double* g, const double* mdiag, double radius, double* d) {
    count(cost_trsub(n));
    double Hs[OR_MAXNC * OR_MAXNC], gs[OR_MAXNC], sc[OR_MAXNC];
    for (int i = 0; i < n; i++) sc[i] = mdiag ? 1.0 / sqrt(mdiag[i]) : 1.0;
    for (int i = 0; i < n; i++) {
        gs[i] = sc[i] * g[i];
        for (int j = 0; j < n; j++) Hs[i * n + j] = sc[i] * H[i * n + j] * sc[j];
    }
    double lam[OR_MAXNC], V[OR_MAXNC * OR_MAXNC], gt[OR_MAXNC], u[OR_MAXNC];
    jacobi_eig(n, Hs, lam, V);
    double lmin = lam[0];
    int imin = 0;
    for (int i = 1; i < n; i++) if (lam[i] < lmin) { lmin = lam[i]; imin = i; }
    for (int k = 0; k < n; k++) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += V[i * n + k] * gs[i];
        gt[k] = s;
    }
    if (lmin > 0.0 && unorm(n, gt, lam, 0.0) <= radius) {
        for (int k = 0; k < n; k++) u[k] = -gt[k] / lam[k];          /* Newton step fits */
    } else {
        double lo = lmin > 0.0 ? 0.0 : -lmin;
        double lo_eff = lo * (1.0 + 1e-15) + 1e-300;
        if (lmin <= 0.0 && unorm(n, gt, lam, lo_eff) < radius) {
            /* hard case: g has no component on the lowest eigenvector;
             * complete the step to the boundary along that eigenvector */
            double s2 = 0.0;
            for (int k = 0; k < n; k++) {
                u[k] = (k == imin) ? 0.0 : -gt[k] / (lam[k] - lmin);
                s2 += u[k] * u[k];
            }
            u[imin] = sqrt(fmax(radius * radius - s2, 0.0));
        } else {
            /* ||u(eta)|| decreases monotonically for eta > lo: bisect */
            double hi = lo + 1.0;
            for (int it = 0; it < 2000 && unorm(n, gt, lam, hi) > radius; it++) hi = lo + 2.0 * (hi - lo);
            for (int it = 0; it < 2000; it++) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                if (unorm(n, gt, lam, mid) > radius) lo = mid; else hi = mid;
            }
            for (int k = 0; k < n; k++) u[k] = -gt[k] / (lam[k] + hi);
        }
    }
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int k = 0; k < n; k++) s += V[i * n + k] * u[k];
        d[i] = sc[i] * s;
    }
    double pred = 0.0;
    for (int i = 0; i < n; i++) {
        double hd = 0.0;
        for (int j = 0; j < n; j++) hd += H[i * n + j] * d[j];
        pred += g[i] * d[i] + 0.5 * d[i] * hd;
    }
    return pred;
}

/* Newton step -H^{-1} g through the eigendecomposition; returns 0 if H is
 * positive definite, -1 otherwise (no step). */
static int newton_step(int n, const double* H, const double* g, double* d) {
    count(add_ops(cost_chol(n), ops(2.0 * n * n, 0, 0, 0, 0)));
    double lam[OR_MAXNC], V[OR_MAXNC * OR_MAXNC];
    jacobi_eig(n, H, lam, V);
    for (int k = 0; k < n; k++) if (!(lam[k] > 0.0)) return -1;
    for (int i = 0; i < n; i++) d[i] = 0.0;
    for (int k = 0; k < n; k++) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += V[i * n + k] * g[i];
        for (int i = 0; i < n; i++) d[i] -= V[i * n + k] * s / lam[k];
    }
    return 0;
}

static double vnorm_m(int n, const double* d, const double* mdiag) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += (mdiag ? mdiag[i] : 1.0) * d[i] * d[i];
    return sqrt(s);
}

/* Dominant eigenvalue acceleration (reading R7).  dk = latest SS update,
 * d1 = the one before.  Applied on every DEM_PERIOD-th update of a run when
 * the updates shrink (||dk|| < ||d1||) and 0 < lambda < 1.
 * Returns the factor lambda / (1 - lambda) to add dk with, or 0. */
#define DEM_PERIOD 3
static double dem_factor(int nc, const double* dk, const double* d1) {
    double n0 = 0.0, n1 = 0.0, p01 = 0.0;
    for (int i = 0; i < nc; i++) {
        n0 += dk[i] * dk[i];
        n1 += d1[i] * d1[i];
        p01 += dk[i] * d1[i];
    }
    if (!(n1 > 0.0) || !(n0 < n1)) return 0.0;
    double lam = p01 / n1;
    if (!(lam > 0.0 && lam < 1.0)) return 0.0;
    return lam / (1.0 - lam);
}

/* ------------------------------------------------------------------------ */
/* Stability analysis (Sec. 2.2.1, Appendix B.1, Alg. 2) for one trial.      */
/* d_i = ln z_i + ln phi_i(z).  lnW holds the trial (in/out).  Returns tm at */
/* the final point; *iters_ss, *iters_tr count updates; flags get ST_* bits. */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lnW[OR_MAXNC];
    double tm;
    int iters_ss, iters_tr;
    int used_tr, maxiter, nonfinite;
} or_trial;

/* tm (reading R2) and grad-tm/dW = ln W + ln phi(W) - d at a trial lnW. */
static int stab_eval(const or_mix* m, const double* d, const double* lnW, or_phase* ph, double* gt, double* tm) {
    int nc = m->nc;
    count(ops(6.0 * nc, 1, 0, nc, 0));
    double W[OR_MAXNC], Wt = 0.0, c[OR_MAXNC];
    for (int i = 0; i < nc; i++) { W[i] = exp(lnW[i]); Wt += W[i]; }
    for (int i = 0; i < nc; i++) c[i] = W[i] / Wt;
    if (or_eos(m, c, ph)) return -1;
    double t = 1.0;
    for (int i = 0; i < nc; i++) {
        gt[i] = lnW[i] + ph->lnphi[i] - d[i];
        t += W[i] * (gt[i] - 1.0);
    }
    *tm = t;
    return isfinite(t) ? 0 : -1;
}

static double maxabs(int n, const double* v) {
    double r = 0.0;
    for (int i = 0; i < n; i++) if (fabs(v[i]) > r || v[i] != v[i]) r = (v[i] != v[i]) ? INFINITY : fabs(v[i]);
    return r;
}

/* Stability trust-region point (Appendix B.1, Eqs. analysis_grad and
 * analysis_hess with reading R4): gradient g_i = sqrt(W_i) gt_i and Hessian
 * H_ij = sqrt(W_i W_j) d ln phi_i / d W_j + delta_ij (1 + g_i / beta_i) in
 * beta = 2 sqrt(W), where g_i / beta_i = gt_i / 2. */
static int stab_point(const or_mix* m, const double* d, const double* lnW, double* gt, double* tm, double* g,
                      double* H) {
    int nc = m->nc;
    or_phase ph;
    if (stab_eval(m, d, lnW, &ph, gt, tm)) return -1;
    double W[OR_MAXNC], Wt = 0.0, c[OR_MAXNC], J[OR_MAXNC * OR_MAXNC];
    for (int i = 0; i < nc; i++) { W[i] = exp(lnW[i]); Wt += W[i]; }
    for (int i = 0; i < nc; i++) c[i] = W[i] / Wt;
    or_dlnphi_dn(m, c, &ph, J);
    count(ops(4.0 * nc * (nc + 1) + 2 * nc, 0, nc, 0, 0));
    for (int i = 0; i < nc; i++) g[i] = sqrt(W[i]) * gt[i];
    for (int i = 0; i < nc; i++)
        for (int j = 0; j < nc; j++)
            H[i * nc + j] = sqrt(W[i] * W[j]) * J[i * nc + j] / Wt + (i == j ? 1.0 + 0.5 * gt[i] : 0.0);
    return 0;
}

/* stop_on_negative = 1 follows the paper (stop at tm < 0); the grading
 * helper passes 0 to converge every trial to its stationary point. */
void or_stability_trial(const or_mix* m, const double* d, or_trial* tr, int stop_on_negative, int kss, int ktr,
                        double tol) {
    int nc = m->nc;
    or_phase ph;
    double gt[OR_MAXNC], tm, dprev[OR_MAXNC] = {0};
    tr->iters_ss = tr->iters_tr = tr->used_tr = tr->maxiter = tr->nonfinite = 0;
    /* successive substitution, Eq. ss_analyser, with DEM (R7): the
     * evaluation after an accelerated update must succeed with a smaller
     * residual, else the plain update is restored. */
    double lnW_plain[OR_MAXNC], res_prev = INFINITY;
    int dem_pending = 0;
    g_stage = 1;
    for (int it = 0;; it++) {
        int bad = stab_eval(m, d, tr->lnW, &ph, gt, &tm);
        double res = bad ? INFINITY : maxabs(nc, gt);
        if (dem_pending && (bad || !(res < res_prev))) {
            dem_pending = 0;
            memcpy(tr->lnW, lnW_plain, sizeof(double) * nc);
            continue;
        }
        dem_pending = 0;
        if (bad) { tr->nonfinite = 1; tr->tm = NAN; return; }
        if (stop_on_negative && tm < -EPS_NEG) { tr->tm = tm; return; }
        if (res < tol) { tr->tm = tm; return; }
        if (it >= kss) break;
        double dk[OR_MAXNC];
        for (int i = 0; i < nc; i++) { dk[i] = -gt[i]; tr->lnW[i] += dk[i]; }
        int s = tr->iters_ss + 1;
        if (s % DEM_PERIOD == 0) {
            double f = dem_factor(nc, dk, dprev);
            if (f > 0.0) {
                memcpy(lnW_plain, tr->lnW, sizeof(double) * nc);
                for (int i = 0; i < nc; i++) tr->lnW[i] += dk[i] * f;
                dem_pending = 1;
                res_prev = res;
            }
        }
        for (int i = 0; i < nc; i++) dprev[i] = dk[i];
        tr->iters_ss = s;
    }
    /* trust region on beta = 2 sqrt(W), Eqs. tr_sa, analysis_grad,
     * analysis_hess (readings R4, R9) */
    tr->used_tr = 1;
    g_stage = 2;
    double beta[OR_MAXNC], g[OR_MAXNC], H[OR_MAXNC * OR_MAXNC];
    double radius = -1.0;
    if (stab_point(m, d, tr->lnW, gt, &tm, g, H)) { tr->nonfinite = 1; tr->tm = NAN; return; }
    for (int i = 0; i < nc; i++) beta[i] = 2.0 * exp(0.5 * tr->lnW[i]);
    for (int it = 0;; it++) {
        if (stop_on_negative && tm < -EPS_NEG) break;
        if (maxabs(nc, g) < tol) break;
        if (it == ktr) { tr->maxiter = 1; break; }
        double step[OR_MAXNC];
        if (radius < 0.0) { /* R9: initial radius */
            if (newton_step(nc, H, g, step) == 0) radius = vnorm_m(nc, step, NULL);
            else radius = 1.0;
        }
        double pred = or_tr_subproblem(nc, H, g, NULL, radius, step);
        double lnWn[OR_MAXNC], gtn[OR_MAXNC], gn[OR_MAXNC], Hn[OR_MAXNC * OR_MAXNC], tmn;
        for (int i = 0; i < nc; i++) {
            double b = fabs(beta[i] + step[i]); /* tm(beta) is even in each beta_i */
            lnWn[i] = 2.0 * log(0.5 * b);
        }
        count(ops(3.0 * nc + 2.0 * nc * nc, 0, 0, 0, nc));
        int bad = stab_point(m, d, lnWn, gtn, &tmn, gn, Hn);
        /* R9: below PRED_TRUST the predicted change is under the rounding
         * of tm itself and the ratio is noise: accept, keep the radius.
         * A trial point that cannot be evaluated is a rejected step. */
        int trusted = fabs(pred) > PRED_TRUST * (1.0 + fabs(tm));
        double rho = bad ? -1.0 : (trusted ? (tmn - tm) / pred : 0.5);
        if (rho > 0.0) {
            for (int i = 0; i < nc; i++) {
                tr->lnW[i] = lnWn[i];
                beta[i] = fabs(beta[i] + step[i]);
                gt[i] = gtn[i];
                g[i] = gn[i];
            }
            memcpy(H, Hn, sizeof(double) * nc * nc);
            tm = tmn;
        }
        if (rho <= 0.25) radius *= 0.5;
        else if (rho >= 0.75) radius *= 2.0;
        tr->iters_tr = it + 1;
    }
    tr->tm = tm;
}

/* K from the stability trials (Sec. 2.2.1, last sentence; reading R16):
 * the trial with the lower tm gives K_i = w_i / z_i (vapour-like) or
 * z_i / w_i (liquid-like), w = W / sum W its composition.  At a stationary
 * point sum W = exp(-tpd) is near 1; a trial stopped at its first negative
 * tm can be far from one. */
static void stab_lnK(int nc, const double* lnz, const or_trial* tv, const or_trial* tl, double* lnK) {
    const or_trial* t = (tl->tm < tv->tm) ? tl : tv;
    double sw = 0.0;
    for (int i = 0; i < nc; i++) sw += exp(t->lnW[i]);
    double ls = log(sw);
    for (int i = 0; i < nc; i++)
        lnK[i] = (t == tl) ? lnz[i] - (t->lnW[i] - ls) : (t->lnW[i] - ls) - lnz[i];
}

/* ------------------------------------------------------------------------ */
/* Phase split (Sec. 2.2.2, Appendix B.2).                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nphase;
    double beta, x[OR_MAXNC], y[OR_MAXNC], K[OR_MAXNC];
    int status;
    int it_split_ss, it_split_tr, it_stab_ss, it_stab_tr;
    double tm_min; /* min tm over the stability trials when run, else NAN */
} or_result;

static void set_single(int nc, const double* z, or_result* r) {
    r->nphase = 1;
    r->beta = 0.0;
    for (int i = 0; i < nc; i++) { r->x[i] = z[i]; r->y[i] = z[i]; r->K[i] = 1.0; }
}

/* x, y from K and theta (Eq. material_balance) */
static void xy_from(int nc, const double* z, const double* K, double th, double* x, double* y) {
    for (int i = 0; i < nc; i++) {
        x[i] = z[i] / (1.0 + th * (K[i] - 1.0));
        y[i] = K[i] * x[i];
    }
}

/* Split evaluation in n^V (Eqs. gibbs, split_grad, split_hess; reading R5). */
typedef struct {
    double th, x[OR_MAXNC], y[OR_MAXNC];
    double gt[OR_MAXNC], G, H[OR_MAXNC * OR_MAXNC], mdiag[OR_MAXNC];
    double ZL, ZV;
} or_splitpt;

static int split_eval(const or_mix* m, const double* z, const double* nV, or_splitpt* s) {
    int nc = m->nc;
    count(ops(12.0 * nc + 5.0 * nc * (nc + 1) + 2.0 * nc * nc, 2 + nc, nc, 0, 2.0 * nc));
    double th = 0.0;
    for (int i = 0; i < nc; i++) th += nV[i];
    s->th = th;
    for (int i = 0; i < nc; i++) {
        s->y[i] = nV[i] / th;
        s->x[i] = (z[i] - nV[i]) / (1.0 - th);
    }
    or_phase pl, pv;
    if (or_eos(m, s->x, &pl) || or_eos(m, s->y, &pv)) return -1;
    s->ZL = pl.Z;
    s->ZV = pv.Z;
    double JL[OR_MAXNC * OR_MAXNC], JV[OR_MAXNC * OR_MAXNC];
    or_dlnphi_dn(m, s->x, &pl, JL);
    or_dlnphi_dn(m, s->y, &pv, JV);
    double G = 0.0;
    for (int i = 0; i < nc; i++) {
        double mul = log(s->x[i]) + pl.lnphi[i], muv = log(s->y[i]) + pv.lnphi[i];
        s->gt[i] = muv - mul;
        G += (z[i] - nV[i]) * mul + nV[i] * muv;
    }
    s->G = G;
    double w = 1.0 / (th * (1.0 - th));
    for (int i = 0; i < nc; i++) {
        s->mdiag[i] = z[i] / (s->x[i] * s->y[i]);
        for (int j = 0; j < nc; j++)
            s->H[i * nc + j] = w * ((i == j ? s->mdiag[i] : 0.0) - 1.0 + th * JL[i * nc + j] + (1.0 - th) * JV[i * nc + j]);
    }
    return isfinite(G) ? 0 : -1;
}

/* 0.99 fraction-to-boundary cut keeping 0 < n^V_i + d_i < z_i (R9) */
static double boundary_cut(int nc, const double* z, const double* nV, const double* d) {
    double tau = 1.0;
    for (int i = 0; i < nc; i++) {
        if (d[i] < 0.0) { double t = 0.99 * nV[i] / (-d[i]); if (t < tau) tau = t; }
        else if (d[i] > 0.0) { double t = 0.99 * (z[i] - nV[i]) / d[i]; if (t < tau) tau = t; }
    }
    return tau;
}

/* Finish a two-phase result: canonical labels (R14), K = y/x. */
static void finish_two_phase(int nc, double th, const double* x, const double* y, double ZL, double ZV, or_result* r) {
    int swap = ZV < ZL;
    r->nphase = 2;
    r->beta = swap ? 1.0 - th : th;
    for (int i = 0; i < nc; i++) {
        r->x[i] = swap ? y[i] : x[i];
        r->y[i] = swap ? x[i] : y[i];
        r->K[i] = r->y[i] / r->x[i];
    }
}

/* Split from ln K: successive substitution (cap kss, DEM R7, convergence
 * R10), then trust region + Newton polish.  it_done counts updates already
 * taken by the caller's run (DEM numbering restarts: fresh cap, R11). */
static void or_split(const or_mix* m, const double* z, double* lnK, or_result* r) {
    int nc = m->nc;
    g_stage = 3;
    double K[OR_MAXNC], x[OR_MAXNC], y[OR_MAXNC], th = 0.5, dprev[OR_MAXNC] = {0};
    or_phase pl, pv;
    r->it_split_ss = 0;
    r->it_split_tr = 0;
    double lnK_plain[OR_MAXNC], res_prev = INFINITY;
    int dem_pending = 0;
    for (int it = 0;; it++) {
        /* 0 ok, 1 collapse (trivial K or no Rachford-Rice root), 2 non-finite */
        int fail = 0;
        double gt[OR_MAXNC], res = INFINITY;
        if (maxabs(nc, lnK) < TRIVIAL_LNK) fail = 1;
        if (!fail) {
            for (int i = 0; i < nc; i++) K[i] = exp(lnK[i]);
            count(ops(6.0 * nc, 0, 0, nc, 0));
            if (or_rr(nc, z, K, &th)) fail = 1;
        }
        if (!fail) {
            xy_from(nc, z, K, th, x, y);
            if (or_eos(m, x, &pl) || or_eos(m, y, &pv)) fail = 2;
        }
        if (!fail) {
            for (int i = 0; i < nc; i++) gt[i] = lnK[i] + pv.lnphi[i] - pl.lnphi[i];
            res = maxabs(nc, gt);
            if (!(res < INFINITY)) fail = 2;
        }
        if (dem_pending && (fail || !(res < res_prev))) {
            dem_pending = 0;
            memcpy(lnK, lnK_plain, sizeof(double) * nc);
            continue;
        }
        dem_pending = 0;
        if (fail == 1) { r->status |= ST_COLLAPSE; set_single(nc, z, r); return; }
        if (fail == 2) { r->status |= ST_NONFINITE; set_single(nc, z, r); return; }
        if (res <= TOL_FUG) {
            if (!(th > 0.0 && th < 1.0)) { r->status |= ST_COLLAPSE; set_single(nc, z, r); return; }
            finish_two_phase(nc, th, x, y, pl.Z, pv.Z, r);
            return;
        }
        if (it >= KSS_SPLIT) break;
        double dk[OR_MAXNC];
        for (int i = 0; i < nc; i++) { dk[i] = -gt[i]; lnK[i] += dk[i]; }
        int s = r->it_split_ss + 1;
        if (s % DEM_PERIOD == 0) {
            double f = dem_factor(nc, dk, dprev);
            if (f > 0.0) {
                memcpy(lnK_plain, lnK, sizeof(double) * nc);
                for (int i = 0; i < nc; i++) lnK[i] += dk[i] * f;
                dem_pending = 1;
                res_prev = res;
            }
        }
        for (int i = 0; i < nc; i++) dprev[i] = dk[i];
        r->it_split_ss = s;
    }
    /* trust region on G in n^V (Eq. newton_splitter), from the last
     * evaluated SS point (theta, x, y of the cap-th evaluation) */
    r->status |= ST_SPLIT_TR;
    g_stage = 4;
    double nV[OR_MAXNC];
    if (th > 0.0 && th < 1.0) {
        for (int i = 0; i < nc; i++) nV[i] = th * y[i];
    } else {
        /* R13: a negative-flash SS endpoint is no feasible start; take the
         * material-balance point of the same K at theta = 1/2 */
        for (int i = 0; i < nc; i++) nV[i] = 0.5 * K[i] * z[i] / (1.0 + 0.5 * (K[i] - 1.0));
    }
    or_splitpt cur, nxt;
    if (split_eval(m, z, nV, &cur)) { r->status |= ST_NONFINITE; set_single(nc, z, r); return; }
    double radius = -1.0;
    int it = 0, phase_newton = 0, newton_steps = 0;
    for (;;) {
        double res = maxabs(nc, cur.gt);
        if (!(cur.th > COLLAPSE_TH && cur.th < 1.0 - COLLAPSE_TH)) {  /* R13 */
            r->status |= ST_MAXITER | ST_COLLAPSE;
            set_single(nc, z, r);
            return;
        }
        if (phase_newton) {
            if (res <= TOL_FUG && newton_steps >= 1) break;
            if (newton_steps == KNEWTON_POLISH) { r->status |= ST_MAXITER; break; }
        } else if (res < TOL_SPLIT_TR) {
            phase_newton = 1;
            continue;
        }
        if (!phase_newton && it == KTR_SPLIT) { r->status |= ST_MAXITER; break; }
        double step[OR_MAXNC];
        if (phase_newton) {
            if (newton_step(nc, cur.H, cur.gt, step)) { /* H not PD: stop polishing */
                if (res > TOL_FUG) r->status |= ST_MAXITER;
                break;
            }
            double tau = boundary_cut(nc, z, nV, step);
            for (int i = 0; i < nc; i++) nV[i] += tau * step[i];
            if (split_eval(m, z, nV, &cur)) { r->status |= ST_NONFINITE; set_single(nc, z, r); return; }
            newton_steps++;
            r->it_split_tr++;
            continue;
        }
        if (radius < 0.0) {
            if (newton_step(nc, cur.H, cur.gt, step) == 0) radius = vnorm_m(nc, step, cur.mdiag);
            else radius = 1.0;
        }
        double pred = or_tr_subproblem(nc, cur.H, cur.gt, cur.mdiag, radius, step);
        double tau = boundary_cut(nc, z, nV, step);
        if (tau < 1.0) {
            for (int i = 0; i < nc; i++) step[i] *= tau;
            pred = 0.0;
            for (int i = 0; i < nc; i++) {
                double hd = 0.0;
                for (int j = 0; j < nc; j++) hd += cur.H[i * nc + j] * step[j];
                pred += cur.gt[i] * step[i] + 0.5 * step[i] * hd;
            }
        }
        double nVn[OR_MAXNC];
        for (int i = 0; i < nc; i++) nVn[i] = nV[i] + step[i];
        int bad = split_eval(m, z, nVn, &nxt);
        int trusted = fabs(pred) > PRED_TRUST * (1.0 + fabs(cur.G));
        double rho = bad ? -1.0 : (trusted ? (nxt.G - cur.G) / pred : 0.5);
        if (rho > 0.0) {
            memcpy(nV, nVn, sizeof(double) * nc);
            cur = nxt;
        }
        if (rho <= 0.25) radius *= 0.5;
        else if (rho >= 0.75) radius *= 2.0;
        it++;
        r->it_split_tr = it;
    }
    if (!(cur.th > 0.0 && cur.th < 1.0)) { r->status |= ST_COLLAPSE; set_single(nc, z, r); return; }
    finish_two_phase(nc, cur.th, cur.x, cur.y, cur.ZL, cur.ZV, r);
}

/* ------------------------------------------------------------------------ */
/* Full plain flash (Sec. 2.2.3 flowchart).                                 */
/* lnK_init == NULL: Wilson initialisation and the 3-iteration precheck.    */
/* ------------------------------------------------------------------------ */
void or_flash_one(const or_sys* s, double P, double T, const double* z, or_result* r) {
    int nc = s->nc;
    g_stage = 0;
    or_mix m;
    or_mix_init(s, P, T, &m);
    count(ops(16.0 * nc, nc, nc, 0, nc)); /* constants, ln z, Wilson */
    memset(r, 0, sizeof(*r));
    r->tm_min = NAN;
    double lnz[OR_MAXNC], d[OR_MAXNC], lnKw[OR_MAXNC], lnK[OR_MAXNC];
    or_phase pz;
    for (int i = 0; i < nc; i++) lnz[i] = log(z[i]);
    if (or_eos(&m, z, &pz)) { r->status |= ST_NONFINITE; set_single(nc, z, r); return; }
    for (int i = 0; i < nc; i++) d[i] = lnz[i] + pz.lnphi[i];
    or_wilson(s, P, T, lnKw);
    memcpy(lnK, lnKw, sizeof(lnK));
    /* precheck: 3 SS iterations (R11) */
    int route_stab = 0;
    {
        double K[OR_MAXNC], x[OR_MAXNC], y[OR_MAXNC], th, gt[OR_MAXNC];
        or_phase pl, pv;
        for (int it = 0; it < NPRECHECK; it++) {
            for (int i = 0; i < nc; i++) K[i] = exp(lnK[i]);
            count(ops(6.0 * nc, 0, 0, nc, 0));
            if (or_rr(nc, z, K, &th) || !(th > 0.0 && th < 1.0)) { route_stab = 1; break; }
            xy_from(nc, z, K, th, x, y);
            if (or_eos(&m, x, &pl) || or_eos(&m, y, &pv)) { route_stab = 1; break; }
            for (int i = 0; i < nc; i++) { gt[i] = lnK[i] + pv.lnphi[i] - pl.lnphi[i]; lnK[i] -= gt[i]; }
        }
        if (!route_stab) {
            /* Eq. tpd on the current phases; Delta G by reading R3 */
            double tx = 0.0, ty = 0.0;
            count(ops(8.0 * nc + 5.0, 0, 0, 0, 2.0 * nc));
            for (int i = 0; i < nc; i++) {
                tx += x[i] * (log(x[i]) + pl.lnphi[i] - d[i]);
                ty += y[i] * (log(y[i]) + pv.lnphi[i] - d[i]);
            }
            double dG = (1.0 - th) * tx + th * ty;
            if (!(tx < -EPS_NEG || ty < -EPS_NEG || dG < -EPS_NEG)) route_stab = 1;
        }
    }
    if (!route_stab) {
        r->status |= ST_PRECHECK_UNSTABLE;
        or_split(&m, z, lnK, r);
        return;
    }
    /* stability analysis from Wilson K (Sec. 2.2.1, Alg. 2) */
    r->status |= ST_STAB_RUN;
    or_trial tv, tl;
    for (int i = 0; i < nc; i++) { tv.lnW[i] = lnz[i] + lnKw[i]; tl.lnW[i] = lnz[i] - lnKw[i]; }
    or_stability_trial(&m, d, &tv, 1, KSS_STAB, KTR_STAB, TOL_STAB);
    or_stability_trial(&m, d, &tl, 1, KSS_STAB, KTR_STAB, TOL_STAB);
    r->it_stab_ss = tv.iters_ss + tl.iters_ss;
    r->it_stab_tr = tv.iters_tr + tl.iters_tr;
    if (tv.used_tr || tl.used_tr) r->status |= ST_STAB_TR;
    if (tv.maxiter || tl.maxiter) r->status |= ST_MAXITER;
    if (tv.nonfinite || tl.nonfinite) { r->status |= ST_NONFINITE; set_single(nc, z, r); return; }
    r->tm_min = tv.tm < tl.tm ? tv.tm : tl.tm;
    if (!(r->tm_min < -EPS_NEG)) { set_single(nc, z, r); return; }
    /* K re-estimate (Sec. 2.2.1, last sentence; reading R16) */
    stab_lnK(nc, lnz, &tv, &tl, lnK);
    or_split(&m, z, lnK, r);
}

/* Grading helper: minimum tpd (Eq. tpd) over both Wilson trials, each
 * converged to its stationary point (no early stop at negative tm, residual
 * 1e-9, larger caps than the method's). */
double or_tpd_min_one(const or_sys* s, double P, double T, const double* z) {
    int nc = s->nc;
    or_mix m;
    or_mix_init(s, P, T, &m);
    double lnz[OR_MAXNC], d[OR_MAXNC], lnKw[OR_MAXNC];
    or_phase pz;
    for (int i = 0; i < nc; i++) lnz[i] = log(z[i]);
    if (or_eos(&m, z, &pz)) return NAN;
    for (int i = 0; i < nc; i++) d[i] = lnz[i] + pz.lnphi[i];
    or_wilson(s, P, T, lnKw);
    double best = INFINITY;
    for (int t = 0; t < 2; t++) {
        or_trial tr;
        for (int i = 0; i < nc; i++) tr.lnW[i] = lnz[i] + (t == 0 ? lnKw[i] : -lnKw[i]);
        or_stability_trial(&m, d, &tr, 0, 60, 200, 1e-9);
        if (tr.nonfinite) continue;
        /* Eq. tpd evaluated at w = W / sum W: second-order accurate in the
         * stationarity residual (unlike -ln sum W) */
        double W[OR_MAXNC], Wt = 0.0, w[OR_MAXNC];
        for (int i = 0; i < nc; i++) { W[i] = exp(tr.lnW[i]); Wt += W[i]; }
        for (int i = 0; i < nc; i++) w[i] = W[i] / Wt;
        or_phase pw;
        if (or_eos(&m, w, &pw)) continue;
        double tpd = 0.0;
        for (int i = 0; i < nc; i++) tpd += w[i] * (log(w[i]) + pw.lnphi[i] - d[i]);
        if (tpd < best) best = tpd;
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Batch entry points (SoA, component-major z[i*n + m]), OpenMP over        */
/* mixtures.  Called through ctypes by the tests and the CPU baseline.      */
/* ------------------------------------------------------------------------ */
static void sys_from(int nc, const double* Tc, const double* Pc, const double* om, const double* kij, or_sys* s) {
    s->nc = nc;
    for (int i = 0; i < nc; i++) { s->Tc[i] = Tc[i]; s->Pc[i] = Pc[i]; s->om[i] = om[i]; }
    for (int i = 0; i < nc * nc; i++) s->kij[i] = kij[i];
}

int oracle_flash_batch(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
                       int64_t n, const double* P, const double* T, const double* z,
                       int32_t* nphase, double* beta, double* x, double* y, double* K,
                       int32_t* status, int32_t* iters, double* tm_min, double* opcount, int nthreads) {
    if (nc < 2 || nc > OR_MAXNC) return -1;
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
    double tot[NSTAGE][NKIND] = {{0}};
#pragma omp parallel num_threads(nthreads)
    {
    memset(g_ops, 0, sizeof(g_ops));
#pragma omp for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; k++) {
        double zz[OR_MAXNC];
        for (int i = 0; i < nc; i++) zz[i] = z[(int64_t)i * n + k];
        or_result r;
        or_flash_one(&s, P[k], T[k], zz, &r);
        nphase[k] = r.nphase;
        beta[k] = r.beta;
        for (int i = 0; i < nc; i++) {
            x[(int64_t)i * n + k] = r.x[i];
            y[(int64_t)i * n + k] = r.y[i];
            K[(int64_t)i * n + k] = r.K[i];
        }
        status[k] = r.status;
        if (iters) iters[k] = (r.it_split_ss & 0xff) | ((r.it_split_tr & 0xff) << 8) | ((r.it_stab_ss & 0xff) << 16) | ((r.it_stab_tr & 0xff) << 24);
        if (tm_min) tm_min[k] = r.tm_min;
    }
#pragma omp critical
    for (int q = 0; q < NSTAGE; q++)
        for (int k = 0; k < NKIND; k++) tot[q][k] += g_ops[q][k];
    }
    if (opcount)
        for (int q = 0; q < NSTAGE; q++)
            for (int k = 0; k < NKIND; k++) opcount[q * NKIND + k] = tot[q][k];
    return 0;
}

int oracle_tpd_min_batch(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
                         int64_t n, const double* P, const double* T, const double* z, double* tpd, int nthreads) {
    if (nc < 2 || nc > OR_MAXNC) return -1;
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; k++) {
        double zz[OR_MAXNC];
        for (int i = 0; i < nc; i++) zz[i] = z[(int64_t)i * n + k];
        tpd[k] = or_tpd_min_one(&s, P[k], T[k], zz);
    }
    return 0;
}

/* Single-point primitives for the pin tests. */
int oracle_mix_consts(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
                      double P, double T, double* Ai, double* Bi) {
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
    or_mix m;
    or_mix_init(&s, P, T, &m);
    for (int i = 0; i < nc; i++) { Ai[i] = m.Ai[i]; Bi[i] = m.Bi[i]; }
    return 0;
}

int oracle_cubic_roots(double A, double B, double* roots) { return or_cubic_roots(A, B, roots); }

int oracle_eos(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
               double P, double T, const double* c, double* Z, double* lnphi, double* J, double* AB) {
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
    or_mix m;
    or_mix_init(&s, P, T, &m);
    or_phase ph;
    if (or_eos(&m, c, &ph)) return -1;
    *Z = ph.Z;
    for (int i = 0; i < nc; i++) lnphi[i] = ph.lnphi[i];
    if (J) or_dlnphi_dn(&m, c, &ph, J);
    if (AB) { AB[0] = ph.A; AB[1] = ph.B; }
    return 0;
}

int oracle_wilson(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
                  double P, double T, double* lnK) {
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
    or_wilson(&s, P, T, lnK);
    return 0;
}

int oracle_rr(int nc, const double* z, const double* K, double* theta) { return or_rr(nc, z, K, theta); }

double oracle_tr_subproblem(int n, const double* H, const double* g, const double* mdiag, double radius, double* d) {
    return or_tr_subproblem(n, H, g, mdiag, radius, d);
}

/* Stability alone (the ptflash_stability contract): label from the paper's
 * trials with early stop; returns stable flag, min tm and K re-estimate. */
int oracle_stability_batch(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
                           int64_t n, const double* P, const double* T, const double* z,
                           int32_t* stable, double* tm_min, double* K, int nthreads) {
    if (nc < 2 || nc > OR_MAXNC) return -1;
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; k++) {
        double zz[OR_MAXNC], lnz[OR_MAXNC], d[OR_MAXNC], lnKw[OR_MAXNC];
        for (int i = 0; i < nc; i++) zz[i] = z[(int64_t)i * n + k];
        or_mix m;
        or_mix_init(&s, P[k], T[k], &m);
        or_phase pz;
        for (int i = 0; i < nc; i++) lnz[i] = log(zz[i]);
        int bad = or_eos(&m, zz, &pz);
        for (int i = 0; i < nc; i++) d[i] = lnz[i] + (bad ? NAN : pz.lnphi[i]);
        or_wilson(&s, P[k], T[k], lnKw);
        or_trial tv, tl;
        for (int i = 0; i < nc; i++) { tv.lnW[i] = lnz[i] + lnKw[i]; tl.lnW[i] = lnz[i] - lnKw[i]; }
        or_stability_trial(&m, d, &tv, 1, KSS_STAB, KTR_STAB, TOL_STAB);
        or_stability_trial(&m, d, &tl, 1, KSS_STAB, KTR_STAB, TOL_STAB);
        double tmin = tv.tm < tl.tm ? tv.tm : tl.tm;
        tm_min[k] = tmin;
        stable[k] = (tmin < -EPS_NEG) ? 0 : 1;
        double lk[OR_MAXNC];
        stab_lnK(nc, lnz, &tv, &tl, lk);
        for (int i = 0; i < nc; i++) K[(int64_t)i * n + k] = exp(lk[i]);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sensitivities of the converged flash (the implicit-function-theorem idea  */
/* the paper applies to Rachford-Rice in Sec. 4.2.2, applied to the whole   */
/* equilibrium).  Parity unpinned by the paper itself (it prints no          */
/* derivative values); pinned in the tests by central finite differences of  */
/* this oracle's flash and by the binary phase rule.                         */
/* ------------------------------------------------------------------------ */

/* d ln phi_i / dP and d ln phi_i / dT at fixed composition c (Appendix A,
 * Eqs. a_i, b_i, alpha_i, lnphi differentiated by hand).  With
 * s = P: d ln A_i = 1/P, d ln B_i = 1/P;
 * s = T: d ln A_i = 2 a'/a - 2/T (a = 1 + m (1 - sqrt(T/Tc)),
 *        a' = -m / (2 sqrt(T Tc))), d ln B_i = -1/T.
 * A_ij = (1 - k_ij) sqrt(A_i A_j) gives dA_ij = A_ij (d ln A_i + d ln A_j)/2;
 * psi_i = sum_j A_ij c_j, A = sum c_i psi_i, B = sum c_i B_i; the root moves
 * with dZ = -(F_A dA + F_B dB) / F_Z on F = Z^3 - Z^2 + (A - B - B^2) Z - AB;
 * ln phi_i = bb_i (Z - 1) - ln(Z - B) + q_i L, bb_i = B_i/B,
 * q_i = (A bb_i - 2 psi_i)/B, L = ln(1 + B/Z). */
void or_dlnphi_dPT(const or_sys* s, double P, double T, const double* c, double* dP, double* dT) {
    int nc = s->nc;
    or_mix m;
    or_mix_init(s, P, T, &m);
    or_phase ph;
    or_eos(&m, c, &ph);
    double A = ph.A, B = ph.B, Z = ph.Z;
    double L = log(1.0 + B / Z);
    double FZ = 3.0 * Z * Z - 2.0 * Z + A - B - B * B, FA = Z - B, FB = -Z - 2.0 * B * Z - A;
    for (int which = 0; which < 2; which++) {
        double lA[OR_MAXNC], lB[OR_MAXNC];
        for (int i = 0; i < nc; i++) {
            if (which == 0) {
                lA[i] = 1.0 / P;
                lB[i] = 1.0 / P;
            } else {
                double mi = 0.480 + 1.574 * s->om[i] - 0.176 * s->om[i] * s->om[i];
                double a = 1.0 + mi * (1.0 - sqrt(T / s->Tc[i]));
                double ap = -mi / (2.0 * sqrt(T * s->Tc[i]));
                lA[i] = 2.0 * ap / a - 2.0 / T;
                lB[i] = -1.0 / T;
            }
        }
        double dpsi[OR_MAXNC], dA = 0.0, dB = 0.0;
        for (int i = 0; i < nc; i++) {
            double t = 0.0;
            for (int j = 0; j < nc; j++) t += m.Aij[i * nc + j] * 0.5 * (lA[i] + lA[j]) * c[j];
            dpsi[i] = t;
        }
        for (int i = 0; i < nc; i++) {
            dA += c[i] * dpsi[i];
            dB += c[i] * m.Bi[i] * lB[i];
        }
        double dZ = -(FA * dA + FB * dB) / FZ;
        double dL = (dB * Z - B * dZ) / (Z * (Z + B));
        double* out = which == 0 ? dP : dT;
        for (int i = 0; i < nc; i++) {
            double bb = m.Bi[i] / B;
            double dbb = (m.Bi[i] * lB[i] * B - m.Bi[i] * dB) / (B * B);
            double q = (A * bb - 2.0 * ph.psi[i]) / B;
            double dq = ((dA * bb + A * dbb - 2.0 * dpsi[i]) * B - (A * bb - 2.0 * ph.psi[i]) * dB) / (B * B);
            out[i] = dbb * (Z - 1.0) + bb * dZ - (dZ - dB) / (Z - B) + dq * L + q * dL;
        }
    }
}

/* Solve M u = r (n x n, row-major) by Gaussian elimination with partial
 * pivoting; returns -1 if a pivot vanishes. */
static int gauss_solve(int n, const double* Min, const double* r, double* u) {
    double M[OR_MAXNC * OR_MAXNC], b[OR_MAXNC];
    memcpy(M, Min, sizeof(double) * n * n);
    memcpy(b, r, sizeof(double) * n);
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (fabs(M[i * n + k]) > fabs(M[p * n + k])) p = i;
        if (!(fabs(M[p * n + k]) > 0.0)) return -1;
        if (p != k) {
            for (int j = 0; j < n; j++) { double t = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; i++) {
            double f = M[i * n + k] / M[k * n + k];
            for (int j = k; j < n; j++) M[i * n + j] -= f * M[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        double t = b[i];
        for (int j = i + 1; j < n; j++) t -= M[i * n + j] * u[j];
        u[i] = t / M[i * n + i];
    }
    return 0;
}

/* Forward Jacobian of the flash result (beta, x, y) with respect to
 * (P, T, z) at a converged result, the feed z read as mole numbers (the
 * result depends on z / sum z only).  Unknowns v = vapour moles, l = z - v;
 * V = sum v = beta S, L = sum l = (1 - beta) S, S = sum z.  Equilibrium
 * g_i = ln y_i + ln phi_i^V(y) - ln x_i - ln phi_i^L(x) = 0 (Eq. eq_cond),
 * so dv = -H^{-1} (dg/dtheta) dtheta with
 *   H = A^V + A^L, A^V = (diag(1/y) - 1 + J^V)/V, A^L = (diag(1/x) - 1 + J^L)/L
 *   (J = n_T d ln phi / dn, the Hessian of G in n^V, reading R5),
 *   dg/dz = -A^L, dg/dP = d ln phi^V/dP - d ln phi^L/dP (same for T);
 * then d beta = (sum dv - beta sum dz)/S, dy = (dv - y sum dv)/V,
 * dx = (dz - dv - x (sum dz - sum dv))/L.
 * Single phase: beta = 0 and x = y = z/S, so dx_i/dz_j = dy_i/dz_j =
 * (delta_ij - z_i/S)/S and the P, T columns vanish.
 * jac: row-major [(1 + 2 nc) x (nc + 2)], rows beta, x_1..x_nc, y_1..y_nc;
 * columns P, T, z_1..z_nc.  Returns 0, or -1 if H is singular. */
int or_flash_jacobian(const or_sys* s, double P, double T, const double* z, int nphase, double beta, const double* x,
                      const double* y, double* jac) {
    int nc = s->nc, nr = 1 + 2 * nc, ncol = nc + 2;
    double S = 0.0;
    for (int i = 0; i < nc; i++) S += z[i];
    for (int k = 0; k < nr * ncol; k++) jac[k] = 0.0;
    if (nphase != 2) {
        for (int i = 0; i < nc; i++)
            for (int j = 0; j < nc; j++) {
                double d = ((i == j ? 1.0 : 0.0) - z[i] / S) / S;
                jac[(1 + i) * ncol + 2 + j] = d;
                jac[(1 + nc + i) * ncol + 2 + j] = d;
            }
        return 0;
    }
    double V = beta * S, Lm = (1.0 - beta) * S;
    or_mix m;
    or_mix_init(s, P, T, &m);
    or_phase pl, pv;
    or_eos(&m, x, &pl);
    or_eos(&m, y, &pv);
    double JL[OR_MAXNC * OR_MAXNC], JV[OR_MAXNC * OR_MAXNC], AL[OR_MAXNC * OR_MAXNC], H[OR_MAXNC * OR_MAXNC];
    or_dlnphi_dn(&m, x, &pl, JL);
    or_dlnphi_dn(&m, y, &pv, JV);
    for (int i = 0; i < nc; i++)
        for (int j = 0; j < nc; j++) {
            double av = ((i == j ? 1.0 / y[i] : 0.0) - 1.0 + JV[i * nc + j]) / V;
            AL[i * nc + j] = ((i == j ? 1.0 / x[i] : 0.0) - 1.0 + JL[i * nc + j]) / Lm;
            H[i * nc + j] = av + AL[i * nc + j];
        }
    double dPL[OR_MAXNC], dTL[OR_MAXNC], dPV[OR_MAXNC], dTV[OR_MAXNC];
    or_dlnphi_dPT(s, P, T, x, dPL, dTL);
    or_dlnphi_dPT(s, P, T, y, dPV, dTV);
    for (int col = 0; col < ncol; col++) {
        double rhs[OR_MAXNC], dv[OR_MAXNC], dz[OR_MAXNC];
        for (int i = 0; i < nc; i++) {
            dz[i] = (col >= 2 && i == col - 2) ? 1.0 : 0.0;
            if (col == 0) rhs[i] = dPV[i] - dPL[i];
            else if (col == 1) rhs[i] = dTV[i] - dTL[i];
            else rhs[i] = -AL[i * nc + (col - 2)];
        }
        if (gauss_solve(nc, H, rhs, dv)) return -1;
        double sdv = 0.0, sdz = 0.0;
        for (int i = 0; i < nc; i++) {
            dv[i] = -dv[i];
            sdv += dv[i];
            sdz += dz[i];
        }
        jac[col] = (sdv - beta * sdz) / S;
        for (int i = 0; i < nc; i++) {
            jac[(1 + i) * ncol + col] = (dz[i] - dv[i] - x[i] * (sdz - sdv)) / Lm;
            jac[(1 + nc + i) * ncol + col] = (dv[i] - y[i] * sdv) / V;
        }
    }
    return 0;
}

int oracle_dlnphi_dPT(int nc, const double* Tc, const double* Pc, const double* om, const double* kij, double P,
                      double T, const double* c, double* dP, double* dT) {
    if (nc < 2 || nc > OR_MAXNC) return -1;
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
    or_dlnphi_dPT(&s, P, T, c, dP, dT);
    return 0;
}

/* Batch of Jacobians at given converged results (component-major arrays
 * [i * n + k]); jac: [n][(1 + 2 nc)(nc + 2)]; ok[k] = 0 or -1 (singular H). */
int oracle_flash_jacobian_batch(int nc, const double* Tc, const double* Pc, const double* om, const double* kij,
                                int64_t n, const double* P, const double* T, const double* z, const int32_t* nphase,
                                const double* beta, const double* x, const double* y, double* jac, int32_t* ok,
                                int nthreads) {
    if (nc < 2 || nc > OR_MAXNC) return -1;
    or_sys s;
    sys_from(nc, Tc, Pc, om, kij, &s);
    int64_t sz = (int64_t)(1 + 2 * nc) * (nc + 2);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t k = 0; k < n; k++) {
        double zz[OR_MAXNC], xx[OR_MAXNC], yy[OR_MAXNC];
        for (int i = 0; i < nc; i++) {
            zz[i] = z[(int64_t)i * n + k];
            xx[i] = x[(int64_t)i * n + k];
            yy[i] = y[(int64_t)i * n + k];
        }
        ok[k] = or_flash_jacobian(&s, P[k], T[k], zz, nphase[k], beta[k], xx, yy, jac + k * sz);
    }
    return 0;
}
