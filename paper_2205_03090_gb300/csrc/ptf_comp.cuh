// ptf_comp.cuh -- host-side component table of the kernels.
#pragma once
#include <cmath>
#include "ptf_device.cuh"

namespace ptf {

struct CompHost {
    int nc;
    double Tc[16], Pc[16], om[16], kij[256];
};

// Component table of the kernels from the host data (Appendix A, Eq. m_i;
// Eq. wilson): 1 - k_ij, m_i = 0.480 + 1.574 w - 0.176 w^2, 5.373 (1 + w).
template <int NC>
Comp<NC> make_comp(const CompHost& h) {
    Comp<NC> c;
    for (int i = 0; i < NC; i++) {
        for (int j = 0; j < NC; j++) {
            c.kk[i * NC + j] = 1.0 - h.kij[i * NC + j];
            c.kkf[i * NC + j] = (float)c.kk[i * NC + j];
        }
        c.Tc[i] = h.Tc[i];
        c.Pc[i] = h.Pc[i];
        c.lnPc[i] = std::log(h.Pc[i]);
        c.mi[i] = 0.480 + 1.574 * h.om[i] - 0.176 * h.om[i] * h.om[i];
        c.wc[i] = kWilson * (1.0 + h.om[i]);
        c.rsTc[i] = 1.0 / std::sqrt(h.Tc[i]);
        c.sOmA[i] = std::sqrt(kOmegaA / h.Pc[i]);
        c.OmB[i] = kOmegaB / h.Pc[i];
    }
    return c;
}

}  // namespace ptf
