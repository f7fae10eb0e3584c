// ptf_adjoint.cuh -- reverse-mode sensitivities of the converged flash.
//
// The paper differentiates the Rachford-Rice root by the implicit-function
// theorem instead of through the iterations (Sec. 4.2.2).  The same idea on
// the whole equilibrium: with the feed z read as mole numbers (results depend
// on z / sum z), vapour moles v, l = z - v, V = sum v = beta S,
// L = sum l = (1 - beta) S, S = sum z, the converged split satisfies
// g(v; P, T, z) = ln y + ln phi^V(y) - ln x - ln phi^L(x) = 0 (Eq. eq_cond),
// so dv = -H^{-1} (dg/dz dz + dg/dP dP + dg/dT dT) with H the Hessian of G in
// n^V (Eq. split_hess, reading R5):
//   H = A^V + A^L, A^V = (diag(1/y) - 1 + J^V)/V, A^L = (diag(1/x) - 1 + J^L)/L,
//   dg/dz = -A^L, dg/dP = d ln phi^V/dP - d ln phi^L/dP (likewise T).
// For an output functional l = gb beta + gx.x + gy.y:
//   dl = a.dv + b.dz,
//   a_i = gb/S + (gy_i - gy.y)/V - (gx_i - gx.x)/L,
//   b_i = -beta gb/S + (gx_i - gx.x)/L,
// and with lambda = H^{-1} a (H symmetric):
//   dl/dz = A^L lambda + b,  dl/dP = -lambda.(dg/dP),  dl/dT = -lambda.(dg/dT).
// One mixture per thread; one Cholesky solve replaces the nc + 2 solves of
// the forward Jacobian.
#pragma once
#include "ptf_kernels.cuh"

namespace ptf {

struct AdjIO {
    int64_t n;
    const double *P, *T, *z;
    const int32_t* nphase;
    const double *beta, *x, *y;
    const double *gb, *gx, *gy;  // upstream gradients (each may be null: zero)
    double *gP, *gT, *gz;
    int32_t* astatus;            // 0 two-phase, 1 single phase, 2 split Hessian not positive definite (may be null)
};

// d ln phi_i / ds at fixed composition c for one parameter s, given
// la_i = d ln sqrt(A_i) / ds and lb_i = d ln B_i / ds.  In the form of eos():
// ln phi_i = B_i u - ln(Z - B) - psi_i v, u = (Z - 1)/B + A L / B^2,
// v = 2 L / B, L = ln(1 + B/Z), psi_i = sqrt(A_i) sum_j (1 - k_ij) sqrt(A_j) c_j.
template <int NC>
__device__ __forceinline__ void dlnphi_ds(const Comp<NC>& cp, const Mix<NC>& mx, const double* c, const Phase<NC>& ph,
                                          const double* la, const double* lb, double* out) {
    const double A = ph.A, B = ph.B, Z = ph.Z, L = ph.L;
    double dpsi[NC], dA = 0.0, dB = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < NC; j++) t = fma(cp.kk[i * NC + j] * mx.sA[j] * la[j], c[j], t);
        dpsi[i] = fma(ph.psi[i], la[i], mx.sA[i] * t);
        dA = fma(c[i], dpsi[i], dA);
        dB = fma(c[i], mx.B[i] * lb[i], dB);
    }
    const double FZ = fma(fma(3.0, Z, -2.0), Z, A - B - B * B), FA = Z - B, FB = -Z - 2.0 * B * Z - A;
    const double dZ = -(FA * dA + FB * dB) / FZ;
    const double dL = (dB * Z - B * dZ) / (Z * (Z + B));
    const double iB = 1.0 / B, iB2 = iB * iB;
    const double u = (Z - 1.0) * iB + A * L * iB2, v = 2.0 * L * iB;
    const double du = dZ * iB - (Z - 1.0) * dB * iB2 + (dA * L + A * dL) * iB2 - 2.0 * A * L * dB * iB2 * iB;
    const double dv = 2.0 * dL * iB - 2.0 * L * dB * iB2;
    const double dlzb = (dZ - dB) / (Z - B);
#pragma unroll
    for (int i = 0; i < NC; i++)
        out[i] = mx.B[i] * lb[i] * u + mx.B[i] * du - dlzb - dpsi[i] * v - ph.psi[i] * dv;
}

template <int NC>
__device__ __forceinline__ void adjoint_item(const Comp<NC>& cp, const AdjIO& a, int64_t m) {
    const int64_t n = a.n;
    double z[NC], gx[NC], gy[NC], S = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        z[i] = a.z[i * n + m];
        S += z[i];
        gx[i] = a.gx ? a.gx[i * n + m] : 0.0;
        gy[i] = a.gy ? a.gy[i * n + m] : 0.0;
    }
    const double gb = a.gb ? a.gb[m] : 0.0;
    if (a.nphase[m] != 2) {
        // x = y = z / S: dl/dz_j = (g_j - sum_i g_i z_i / S) / S, g = gx + gy
        double gz0 = 0.0;
#pragma unroll
        for (int i = 0; i < NC; i++) gz0 = fma(gx[i] + gy[i], z[i], gz0);
        gz0 /= S;
#pragma unroll
        for (int i = 0; i < NC; i++) a.gz[i * n + m] = (gx[i] + gy[i] - gz0) / S;
        a.gP[m] = 0.0;
        a.gT[m] = 0.0;
        if (a.astatus) a.astatus[m] = 1;
        return;
    }
    const double P = a.P[m], T = a.T[m], beta = a.beta[m];
    const double V = beta * S, L = (1.0 - beta) * S, iV = 1.0 / V, iL = 1.0 / L;
    double x[NC], y[NC];
#pragma unroll
    for (int i = 0; i < NC; i++) {
        x[i] = a.x[i * n + m];
        y[i] = a.y[i * n + m];
    }
    Mix<NC> mx;
    mix_init<NC>(cp, P, T, mx);
    Phase<NC> pl, pv;
    eos<NC>(cp, mx, x, pl);
    eos<NC>(cp, mx, y, pv);
    double JL[NC * (NC + 1) / 2], H[NC * (NC + 1) / 2];
    dlnphi_dn<NC>(cp, mx, x, pl, JL);
    dlnphi_dn<NC>(cp, mx, y, pv, H);
#pragma unroll
    for (int i = 0; i < NC; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const int k = tri(i, j);
            JL[k] = ((i == j ? 1.0 / x[i] : 0.0) - 1.0 + JL[k]) * iL;  // A^L
            H[k] = ((i == j ? 1.0 / y[i] : 0.0) - 1.0 + H[k]) * iV + JL[k];
        }
    double gxx = 0.0, gyy = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        gxx = fma(gx[i], x[i], gxx);
        gyy = fma(gy[i], y[i], gyy);
    }
    double lam[NC], b[NC];
#pragma unroll
    for (int i = 0; i < NC; i++) {
        lam[i] = gb / S + (gy[i] - gyy) * iV - (gx[i] - gxx) * iL;
        b[i] = -beta * gb / S + (gx[i] - gxx) * iL;
    }
    double Lf[NC * (NC + 1) / 2], dfail;
    if (cholesky<NC>(H, 0.0, Lf, &dfail) >= 0) {
#pragma unroll
        for (int i = 0; i < NC; i++) a.gz[i * n + m] = NAN;
        a.gP[m] = NAN;
        a.gT[m] = NAN;
        if (a.astatus) a.astatus[m] = 2;
        return;
    }
    fwd<NC>(Lf, lam);
    bwd<NC>(Lf, lam);
    // dl/dz = A^L lambda + b
    for (int i = 0; i < NC; i++) {
        double t = b[i];
        for (int j = 0; j < NC; j++) t = fma(JL[i >= j ? tri(i, j) : tri(j, i)], lam[j], t);
        a.gz[i * n + m] = t;
    }
    // d ln sqrt(A_i) and d ln B_i per unit P and T (Appendix A, Eqs. a_i, b_i, alpha_i)
    double la[NC], lb[NC], dL_[NC], dV_[NC];
    const double iP = 1.0 / P, iT = 1.0 / T;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        la[i] = 0.5 * iP;
        lb[i] = iP;
    }
    dlnphi_ds<NC>(cp, mx, x, pl, la, lb, dL_);
    dlnphi_ds<NC>(cp, mx, y, pv, la, lb, dV_);
    double gP = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) gP = fma(-lam[i], dV_[i] - dL_[i], gP);
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double sq = sqrt(T * cp.Tc[i]);
        const double ai = 1.0 + cp.mi[i] * (1.0 - sqrt(T / cp.Tc[i]));
        la[i] = -cp.mi[i] / (2.0 * sq * ai) - iT;
        lb[i] = -iT;
    }
    dlnphi_ds<NC>(cp, mx, x, pl, la, lb, dL_);
    dlnphi_ds<NC>(cp, mx, y, pv, la, lb, dV_);
    double gT = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) gT = fma(-lam[i], dV_[i] - dL_[i], gT);
    a.gP[m] = gP;
    a.gT[m] = gT;
    if (a.astatus) a.astatus[m] = 0;
}

template <int NC>
__global__ void __launch_bounds__(128, 1) k_adjoint(const __grid_constant__ Comp<NC> cp, AdjIO a) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < a.n; m += (int64_t)gridDim.x * blockDim.x)
        adjoint_item<NC>(cp, a, m);
}

template <int NC>
cudaError_t launch_adjoint(const CompHost& h, const AdjIO& a, int grid, cudaStream_t s) {
    const Comp<NC> cp = make_comp<NC>(h);
    k_adjoint<NC><<<grid, 128, 0, s>>>(cp, a);
    return cudaGetLastError();
}

}  // namespace ptf
