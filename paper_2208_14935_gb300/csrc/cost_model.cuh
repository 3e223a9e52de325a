// Engine selection of Sec. V-A (Eq. 1-3 and the selection rule), shared by
// the planning kernels.  RTT = 1; alpha, beta, gamma are rationals over
// kParamDen, so every comparison is exact in 128-bit integers.
#pragma once

#include "common.cuh"

namespace hytg {

__device__ __forceinline__ int decide_route_counts(unsigned int p, unsigned long long Ei,
                                                   unsigned long long A, unsigned long long Ae,
                                                   unsigned long long L, const CostParams &cp) {
    if (Ae == 0) return kRouteNone;
    const bool resident = p < cp.n_cached;
    if (cp.force_route == kRouteCache && resident) return kRouteCache;
    if (cp.force_route == kRouteF || cp.force_route == kRouteC || cp.force_route == kRouteZ)
        return cp.force_route;
    if (cp.force_route == 5) {
        const unsigned long long h =
            mix64(cp.seed ^ mix64(((unsigned long long)cp.iteration << 32) | p));
        if (resident) return 1 + (int)(h % 4ull);   // cache, F, C, Z
        return 2 + (int)(h % 3ull);                 // F, C, Z
    }
    if (resident) return kRouteCache;
    typedef unsigned __int128 u128;
    const unsigned long long den = cp.m * cp.MR;
    const u128 Tef = ((u128)Ei * cp.d1 + den - 1) / den;
    const u128 Tec = ((u128)Ae * cp.d1 + (u128)A * cp.d2 + den - 1) / den;
    const u128 Tl = ((u128)L + cp.MR - 1) / cp.MR;
    // Tiz = Tl * (gamma + (1 - gamma) * Ae / Ei) = TizN / TizD
    const u128 TizN = Tl * ((u128)cp.gamma_num * Ei + (u128)(kParamDen - cp.gamma_num) * Ae);
    const u128 TizD = (u128)kParamDen * Ei;
    const bool c1 = (u128)kParamDen * Tec < (u128)cp.alpha_num * Tef;
    const bool c2 = (u128)kParamDen * Tec * TizD < (u128)cp.beta_num * TizN;
    if (c1 && c2) return kRouteC;
    if (Tef * TizD < TizN) return kRouteF;
    return kRouteZ;
}

}  // namespace hytg
