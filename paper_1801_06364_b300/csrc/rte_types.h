// rte_types.h -- plain structs shared by the host planning code and the
// device kernels (no device code here, so host compilers can include it).
#pragma once

namespace rte {

// Radix sequence of one transform length (host-built, passed by value).
struct FftPlan {
    int n;
    int npass;
    int radix[12];
};

// Up to six couplings of one output moment (Eq. 6 / Eq. 10).
// type 0: coef * Dz[src];  type 1: coef * (i kx + ky) psi~[src];
// type 2: coef * (i kx - ky) psi~[src]; types 3 and 4: as 1 and 2 with
// psi~[src] replaced by conj(psi~[src](-kx, -ky)) (real-radiance layout).
struct CouplingRow {
    int n;
    int src[6];
    int type[6];
    double coef[6];
};

}  // namespace rte
