// Several lanes per trust-region run.
//
// A trust-region run is a chain of dependent FP64 evaluations.  Once a
// trust-region queue has drained, a persistent kernel ends with a few runs
// per warp, and an FP64 warp instruction costs the SM sub-partition's FP64
// pipe as long with one active lane as with 32.  There a group of G lanes
// (G a power of two >= nc) takes each run, lane r holding component r: the
// O(nc) and O(nc^2) parts of an evaluation (mixing sums, ln phi, n_T d ln phi
// / dn rows, the Hessian, the Cholesky updates, the forward solve) then take
// one or nc instructions instead of nc or nc^2, and 32 / G runs share each
// instruction.
//
// Every group computes exactly what one lane computes, operation for
// operation in the same order: a sum over components gathers the terms with
// shuffles and runs the one-lane chain on every lane of the group; the
// Cholesky factor and the forward solve update entries in the one-lane order
// (right-looking over columns is the same sequence of operations per entry);
// the backward solve gathers the factor's columns and runs the one-lane chain.
// So the several-lanes evaluation reproduces the one-lane results bit for bit
// (the shared expressions are the same inline helpers), and every decision
// is the same on every lane of a group: the scalars all come from identical
// chains, so a group's lanes never diverge around a shuffle.
//
// No dynamic index ever selects a register array entry: a lane picks its row
// out of a per-component array by a predicated scan (pick_row).
#pragma once
#include "ptf_device.cuh"

namespace ptf {

// lanes per run: a power of two >= nc (nc >= 5 only: smaller systems have
// short trips)
template <int NC>
struct GroupLanes {
    static constexpr int G = NC <= 8 ? 8 : 16;
    static constexpr bool ok = NC >= 5 && NC <= 16;
};

struct Grp {
    unsigned mask;  // the lanes of this lane's group
    int r;          // this lane's component within the group (>= NC: a padding lane)
};

template <int G>
__device__ __forceinline__ Grp make_grp() {
    const int lane = threadIdx.x & 31;
    Grp g;
    g.r = lane & (G - 1);
    g.mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    return g;
}

// value v of the group's lane k
template <int G>
__device__ __forceinline__ double gat(const Grp& g, double v, int k) {
    return __shfl_sync(g.mask, v, k, G);
}

// a[r] without a dynamic register index
template <int NC>
__device__ __forceinline__ double pick_row(const double* a, int r) {
    double v = a[0];
#pragma unroll
    for (int j = 1; j < NC; j++)
        if (j == r) v = a[j];
    return v;
}

// max |v_i| over the group's components, NaN -> infinity (as maxabs)
template <int NC, int G>
__device__ __forceinline__ double gmaxabs(const Grp& g, double v) {
    double r = 0.0;
    bool nan = false;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double vi = gat<G>(g, v, i);
        r = fmax(r, fabs(vi));
        nan |= vi != vi;
    }
    return nan ? INFINITY : r;
}

// sum_i a_i b_i as the one-lane chain acc = fma(a_i, b_i, acc), i ascending
template <int NC, int G>
__device__ __forceinline__ double gdot(const Grp& g, double a, double b, double acc) {
#pragma unroll
    for (int i = 0; i < NC; i++) acc = fma(gat<G>(g, a, i), gat<G>(g, b, i), acc);
    return acc;
}

// ---------------------------------------------------------------------------
// Phase evaluation (Eqs. mixing_rule, cubic_Z, lnphi) with lane r holding
// component r: psi_r and ln phi_r on their lane, A, B, Z, L on every lane.
// ---------------------------------------------------------------------------
struct PhaseG {
    double A, B, Z, L, psi, lnphi;
};

// kkr: row r of 1 - k_ij; sA, Bi, c: component r's sqrt(A_i), B_i and mole fraction
template <int NC, int G>
__device__ __forceinline__ void eos_g(const Grp& g, const double* kkr, double sA, double Bi, double c, PhaseG& ph) {
    const double sc = sA * c;
    double acc = sc;  // k_ii = 0
#pragma unroll
    for (int j = 0; j < NC; j++) {
        const double scj = gat<G>(g, sc, j);
        if (j != g.r) acc = fma(kkr[j], scj, acc);
    }
    ph.psi = sA * acc;
    double A = 0.0, B = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double ci = gat<G>(g, c, i);
        A = fma(ci, gat<G>(g, ph.psi, i), A);
        B = fma(ci, gat<G>(g, Bi, i), B);
    }
    const Root rt = cubic_select(A, B);
    double u, v;
    lnphi_coef(A, B, rt, u, v);
    ph.lnphi = lnphi_row(Bi, ph.psi, u, v, rt.lzb);
    ph.A = A;
    ph.B = B;
    ph.Z = rt.Z;
    ph.L = rt.L;
}

// Row r of n_T d ln phi / dn, lower part: J[j] for j <= r (Appendix A).
template <int NC, int G>
__device__ __forceinline__ void dlnphi_dn_g(const Grp& g, const double* kkr, double sA, double Bi, const PhaseG& ph,
                                            double* J) {
    const DlnPre<double> c = dln_prelude<double>(ph.A, ph.B, ph.Z, ph.L);
    const DlnVec<double> v = dln_vec<double>(c, Bi, ph.psi, sA);
#pragma unroll
    for (int j = 0; j < NC; j++) {
        const double pj = gat<G>(g, v.p, j), wj = gat<G>(g, v.w, j), Lj = gat<G>(g, v.Lk, j), qj = gat<G>(g, v.q, j),
                     sAj = gat<G>(g, sA, j);
        const double ah1 = (j == g.r) ? v.sAc : mul_rn<double>(kkr[j], v.sAc);  // cL Ahat_rj = ah1 sA_j
        if (j <= g.r) J[j] = dln_entry<double>(v.bb, ph.psi, v.e, v.si, pj, wj, Lj, qj, ah1, sAj);
    }
}

// Fill the upper part of a symmetric matrix's rows from the lower part:
// row r gets H[i] = H_ir (j = r < i) from lane i.
template <int NC, int G>
__device__ __forceinline__ void sym_fill(const Grp& g, double* H) {
#pragma unroll
    for (int i = 1; i < NC; i++) {
#pragma unroll
        for (int j = 0; j < i; j++) {
            const double v = gat<G>(g, H[j], i);
            if (g.r == j) H[i] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Dense linear algebra on a matrix held by rows (lane r: row r).
// ---------------------------------------------------------------------------

// Cholesky of (H + eta I) as `cholesky`: a[] gets row r of the factor, L_rj
// below the diagonal and 1 / L_rr on it.  Column j's pivot is lane j's
// diagonal after the updates of the columns before it; each entry receives
// its updates in the one-lane order.  Returns -1 if positive definite, else
// the failing column (its pivot in dfail); the same on every lane.
template <int NC, int G>
__device__ __forceinline__ int cholesky_g(const Grp& g, const double* H, double eta, double* a, double& dfail) {
#pragma unroll
    for (int j = 0; j < NC; j++) a[j] = (j == g.r) ? H[j] + eta : H[j];
#pragma unroll
    for (int j = 0; j < NC; j++) {
        const double d = gat<G>(g, a[j], j);
        if (!(d > 0.0)) {
            dfail = d;
            return j;
        }
        const double inv = rsqrt_r<double>(d);
        if (g.r == j) a[j] = inv;
        else if (g.r > j) a[j] = a[j] * inv;
#pragma unroll
        for (int c = j + 1; c < NC; c++) {
            const double Lcj = gat<G>(g, a[j], c);
            if (g.r >= c) a[c] = fma(-a[j], Lcj, a[c]);
        }
    }
    return -1;
}

// Solve L y = b in place (b: this lane's row), as `fwd`
template <int NC, int G>
__device__ __forceinline__ double fwd_g(const Grp& g, const double* a, double b) {
#pragma unroll
    for (int k = 0; k < NC; k++) {
        if (g.r == k) b = b * a[k];
        const double yk = gat<G>(g, b, k);
        if (g.r > k) b = fma(-a[k], yk, b);
    }
    return b;
}

// Solve L^T x = b (b: this lane's row), as `bwd`: the one-lane chain on every
// lane, the factor's column i gathered from the lanes below
template <int NC, int G>
__device__ __forceinline__ double bwd_g(const Grp& g, const double* a, double b) {
    double x[NC];
#pragma unroll
    for (int i = NC - 1; i >= 0; i--) {
        double s = gat<G>(g, b, i);
#pragma unroll
        for (int k = i + 1; k < NC; k++) s = fma(-gat<G>(g, a[i], k), x[k], s);
        x[i] = s * gat<G>(g, a[i], i);
    }
    return pick_row<NC>(x, g.r);
}

// As `shift_bound` after a failure at column j (the same on every lane)
template <int NC, int G>
__device__ __forceinline__ double shift_bound_g(const Grp& g, const double* a, int j, double d, double eta) {
    double w[NC], wn = 1.0;
#pragma unroll
    for (int i = NC - 1; i >= 0; i--) {
        const double Lji = gat<G>(g, a[i], j);
        const double Lii = gat<G>(g, a[i], i);
        double s = -Lji;
#pragma unroll
        for (int k = i + 1; k < NC; k++) {
            const double Lki = gat<G>(g, a[i], k);
            if (k < j) s = fma(-Lki, w[k], s);
        }
        w[i] = s * Lii;
        if (i < j) wn = fma(w[i], w[i], wn);
    }
    return eta - d / wn;
}

// As shift_bracket, H and gs by rows (the same chains on every lane)
template <int NC, int G>
__device__ __forceinline__ void shift_bracket_g(const Grp& g, const double* H, double gs, double radius, double eta_lo,
                                                TRShift& sh) {
    double rs = 0.0;
#pragma unroll
    for (int j = 0; j < NC; j++) rs += fabs(H[j]);
    const double hd = pick_row<NC>(H, g.r);
    double gn = 0.0, hn1 = 0.0, mind = 1e300;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double gi = gat<G>(g, gs, i);
        gn = fma(gi, gi, gn);
        hn1 = fmax(hn1, gat<G>(g, rs, i));
        mind = fmin(mind, gat<G>(g, hd, i));
    }
    gn = sqrt(gn);
    sh.elo = fmax(fmax(0.0, eta_lo), fmax(-mind, gn / radius - hn1));
    sh.ehi = gn / radius + hn1;
    sh.active = 1;
    sh.it = 0;
}

// The trust-region subproblem as `tr_shift_step` (FP64), with H, gs and u by
// rows.  Every branch rests on values that are the same on every lane.
template <int NC, int G>
__device__ __forceinline__ int tr_shift_step_g(const Grp& g, const double* H, double gs, double& radius, double eta_lo,
                                               bool newton_only, TRShift& sh, double* a, double& u) {
    constexpr double kShiftTol = 1e-4;
    constexpr double kPoleTol = 1e-12;
    if (sh.active && sh.it > kTRShiftCap + 2) {
        sh.active = 0;
        return -1;
    }
    if (!sh.active && !newton_only && sh.warm > 0.0 && radius > 0.0) {
        shift_bracket_g<NC, G>(g, H, gs, radius, eta_lo, sh);
        sh.zero = 0;
        sh.eta = fmin(fmax(sh.warm, sh.elo), sh.ehi);
    }
    const double eta = sh.active ? sh.eta : 0.0;
    double dfail = 0.0;
    const int jf = cholesky_g<NC, G>(g, H, eta, a, dfail);
    const bool pd = jf < 0;
    double un = 0.0, ur = 0.0;
    if (pd) {
        ur = bwd_g<NC, G>(g, a, fwd_g<NC, G>(g, a, -gs));
        u = ur;
        if (newton_only) return 1;
        un = gdot<NC, G>(g, u, u, 0.0);
        un = sqrt(un);
        if (!sh.active) {
            if (radius <= 0.0) radius = un;
            if (un <= radius) {
                sh.eta = 0.0;
                sh.warm = 0.0;
                return 1;
            }
        } else if (eta == 0.0 && un <= radius) {
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
        shift_bracket_g<NC, G>(g, H, gs, radius, eta_lo, sh);
        sh.zero = 1;
    }
    sh.it++;
    if (!pd) {
        sh.elo = fmax(sh.elo, shift_bound_g<NC, G>(g, a, jf, dfail, eta));
        if (!(sh.ehi > sh.elo)) sh.ehi = 2.0 * sh.elo + 1e-300;
        sh.eta = sh.it >= kTRShiftCap ? sh.ehi
                                      : fmax(sqrt(fmax(sh.elo, 1e-300) * sh.ehi), sh.elo + 1e-3 * (sh.ehi - sh.elo));
        return 0;
    }
    if (!(sh.ehi > sh.elo)) sh.ehi = 2.0 * sh.elo + 1e-300;
    if (un < radius) sh.ehi = eta;
    else sh.elo = fmax(sh.elo, eta);
    if (un < radius && !sh.zero && sh.elo == 0.0) {
        sh.zero = 1;
        sh.eta = 0.0;
        return 0;
    }
    if (sh.ehi - sh.elo <= kPoleTol * sh.ehi) {
        sh.active = 0;
        sh.eta = eta;
        sh.warm = eta;
        return 1;
    }
    const double q = fwd_g<NC, G>(g, a, ur);
    const double qn = gdot<NC, G>(g, q, q, 0.0);
    double en = eta + (un * un / qn) * (un - radius) / radius;
    if (un > radius) en = fmax(en, sh.elo);
    if (!(en >= sh.elo && en < sh.ehi)) {
        en = fmax(sqrt(fmax(sh.elo, 1e-300) * sh.ehi), sh.elo + 1e-3 * (sh.ehi - sh.elo));
    }
    if (en == eta) {
        sh.active = 0;
        sh.eta = eta;
        sh.warm = eta;
        return 1;
    }
    sh.eta = en;
    return 0;
}

}  // namespace ptf
