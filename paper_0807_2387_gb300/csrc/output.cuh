// Output of a 2D plan in the caller's order and physical units (step 8): target k of the cell
// order is target perm[k] of the caller, phi = phi~ + (log s / 2 pi)(sum q - coincident q) and
// H = -s grad phi~ (the torus scaling x -> s x of the plan), in FP64 or FP32 as the caller asks.
#pragma once

#include <stdint.h>

namespace fs {

__device__ __forceinline__ void write_output(int64_t i, double phi, double hx, double hy, void *__restrict__ phi_out,
                                             void *__restrict__ H_out, int out_is_f64)
{
    if (out_is_f64) {
        if (phi_out)
            ((double *)phi_out)[i] = phi;
        if (H_out) {
            ((double *)H_out)[2 * i] = hx;
            ((double *)H_out)[2 * i + 1] = hy;
        }
    } else {
        if (phi_out)
            ((float *)phi_out)[i] = (float)phi;
        if (H_out) {
            ((float *)H_out)[2 * i] = (float)hx;
            ((float *)H_out)[2 * i + 1] = (float)hy;
        }
    }
}

// phi~ and grad phi~ of target k (working precision) -> the caller's outputs at perm[k].
template <typename real>
__device__ __forceinline__ void output_point(int64_t k, real phi_t, real gx_t, real gy_t, real coinc_k,
                                             const int *__restrict__ perm, double shift, double q_sum, double s,
                                             void *__restrict__ phi_out, void *__restrict__ H_out, int out_is_f64)
{
    write_output(perm[k], (double)phi_t + shift * (q_sum - (double)coinc_k), -s * (double)gx_t, -s * (double)gy_t,
                 phi_out, H_out, out_is_f64);
}

}  // namespace fs
