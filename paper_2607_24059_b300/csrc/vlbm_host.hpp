// Host-side helpers shared by the library's translation units (not exported).
#pragma once

#include <cmath>

#include "vlbm.h"
#include "vlbm_device.cuh"

namespace vlbm {

// Bytes of a moving population (all populations, except in the mixed layouts
// whose rest populations are FP32).
inline int elem_bytes(int precision) {
    switch (precision) {
        case VLBM_FP64: return 8;
        case VLBM_FP32: return 4;
        case VLBM_FP16_SHIFTED:
        case VLBM_BF16_SHIFTED:
        case VLBM_FP16_SPLIT:
        case VLBM_BF16_SPLIT: return 2;
        default: return 0;
    }
}

inline bool is_split(int precision) { return precision == VLBM_FP16_SPLIT || precision == VLBM_BF16_SPLIT; }

template <class C>
inline Coef<C> make_coef(const vlbm_params& p, const vlbm_derived& d, const double* scale) {
    Coef<C> k{};
    const int F = p.dim + 1;
    for (int f = 0; f < kMaxFields; ++f) {
        const double om = f < F ? p.omega[f] : 1.0;
        const double al = f < F ? d.alpha[f] : 0.0;
        k.om[f] = (C)om;
        k.al[f] = (C)al;
        k.scale[f] = (C)scale[f];
        k.inv_scale[f] = (C)(1.0 / scale[f]);
    }
    k.i2m = (C)(1.0 / (2.0 * p.mu));
    k.rho_bar = (C)p.rho_bar;
    k.p_bar = (C)std::pow(p.rho_bar, p.gamma);
    k.gamma = (C)p.gamma;
    k.gamma_one = p.gamma == 1.0;
    for (int f = 0; f < kMaxFields; ++f) k.al_s[f] = (C)((f < F ? d.alpha[f] : 0.0) * scale[f]);
    k.i2m_s = (C)(scale[0] / (2.0 * p.mu));
    auto pair = [](double v) { return float2{(float)v, (float)v}; };
    for (int f = 0; f < kMaxFields; ++f) {
        const float al_s = (float)((f < F ? d.alpha[f] : 0.0) * scale[f]);
        const float w = (float)(1.0 - (f < F ? p.omega[f] : 1.0));
        k.p_al[f] = pair(al_s);
        k.p_nal4[f] = pair(-4.0f * al_s);
        k.p_w[f] = pair(w);
        k.p_nwal[f] = pair(-(double)w * al_s);
    }
    k.p_i2m = pair((float)(scale[0] / (2.0 * p.mu)));
    k.p_rho_bar = pair(p.rho_bar);
    k.p_inv_s = pair((float)(1.0 / scale[0]));
    return k;
}


// Storage scales of the shifted half formats: the stored value is g * scale_k,
// chosen so that the deviations of each field sit near unit magnitude.  The rho
// field deviates by O(dx^2 phi) (Prop. 1); a momentum field by O(dx |q|).
inline void vlbm_storage_scales(const vlbm_params& p, double* scale) {
    for (int k = 0; k < 4; ++k) scale[k] = 1.0;
    if (elem_bytes(p.precision) != 2) return;
    scale[0] = 1.0 / (p.dx * p.dx);
    // shifted populations of a momentum field are O(dx |q|); the split layout's
    // non-equilibrium parts are O(dx^2) in every field
    for (int k = 1; k < 4; ++k) scale[k] = is_split(p.precision) ? 1.0 / (p.dx * p.dx) : 1.0 / p.dx;
}


}  // namespace vlbm
