// The image update that closes a subiteration, applied where the back
// projection bp = H_m^T r of a voxel is complete (gather epilogues and the
// stand-alone update kernel).  Preconditioned gradient ascent, Eq. (PGA) with
// the Table 1 preconditioners:
//   OSEM      x <- x bp / sens_m                          (sens_m > 0, else x)
//   OSMAPOSL  x <- x bp / (sens_m + beta_n grad V)        (denominator > 0, else x)
//   BSREM     x <- max(0, x + step x / sens_all (bp - sens_m - beta_n grad V))
//             with step = alpha_t / c_n = alpha_t M       (sens_all > 0, else x)
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace spect {

__device__ __forceinline__ float update1(const UpdateSpec& u, float f, float bp, float sv, float gv, float sa)
{
    switch (u.mode) {
        case kUpdOsem: return sv > 0.f ? f * bp / sv : f;
        case kUpdOsl: {
            const float den = sv + u.beta_n * gv;
            return den > 0.f ? f * bp / den : f;
        }
        case kUpdBsrem: {
            if (!(sa > 0.f)) return f;
            const float v = f + u.step * f / sa * ((bp - sv) - u.beta_n * gv);
            return v > 0.f ? v : 0.f;
        }
        default: return f;
    }
}

// Float4 i4 of a volume: x holds the current image, bp the back projection,
// sv the subset sensitivity (loaded by the caller).
__device__ __forceinline__ float4 update4_sv(const UpdateSpec& u, float4 x, float4 bp, float4 sv, size_t i4)
{
    if (u.bp_add) {
        const float4 b2 = __ldg(reinterpret_cast<const float4*>(u.bp_add) + i4);
        bp = make_float4(bp.x + b2.x, bp.y + b2.y, bp.z + b2.z, bp.w + b2.w);
    }
    float4 gv = make_float4(0.f, 0.f, 0.f, 0.f), sa = gv;
    if (u.grad) gv = __ldg(reinterpret_cast<const float4*>(u.grad) + i4);
    if (u.sens_all) sa = __ldg(reinterpret_cast<const float4*>(u.sens_all) + i4);
    return make_float4(update1(u, x.x, bp.x, sv.x, gv.x, sa.x), update1(u, x.y, bp.y, sv.y, gv.y, sa.y),
                       update1(u, x.z, bp.z, sv.z, gv.z, sa.z), update1(u, x.w, bp.w, sv.w, gv.w, sa.w));
}

__device__ __forceinline__ float4 update4(const UpdateSpec& u, float4 x, float4 bp, size_t i4)
{
    return update4_sv(u, x, bp, __ldg(reinterpret_cast<const float4*>(u.sens) + i4), i4);
}

}  // namespace spect
