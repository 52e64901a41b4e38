// Exact conversion of packed 4/8-bit complex samples to fp16, shared by the fused
// tensor-core kernel's converter warps and the standalone unpack kernel.
//
// fp16(1024 + u) has the bit pattern 0x6400 | u for 0 <= u < 1024.  For two samples taken
// from byte lane `sel` of words a and b, (r & 0x00FF00FF) ^ flip both inserts the 0x64
// exponent bytes and turns each two's-complement byte (or nibble) into u = x + offset; one
// half2 subtraction of 1024 + offset then leaves x exactly.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cstdint>

namespace corr {
namespace conv {

__device__ __forceinline__ uint32_t pair_to_half2(uint32_t a, uint32_t b, uint32_t sel, uint32_t flip, __half2 bias) {
    uint32_t r = (__byte_perm(a, b, sel) & 0x00FF00FFu) ^ flip;
    __half2 h = __hsub2(*reinterpret_cast<__half2*>(&r), bias);
    return *reinterpret_cast<uint32_t*>(&h);
}

// byte-permute selector placing byte k of a in byte 0 and byte k of b in byte 2
__device__ __forceinline__ uint32_t lane_selector(int k) {
    return (uint32_t)(k | (k << 4) | ((k + 4) << 8) | ((k + 4) << 12));
}

// 8-bit samples: flip the sign bit of each byte, bias 1024 + 128
__device__ __forceinline__ __half2 bias8() {
    return __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));   // 1152
}
constexpr uint32_t kFlip8 = 0x64806480u;

// 4-bit samples (one nibble per byte lane after masking): flip bit 3, bias 1024 + 8
__device__ __forceinline__ __half2 bias4() {
    return __halves2half2(__ushort_as_half(0x6408), __ushort_as_half(0x6408));   // 1032
}
constexpr uint32_t kFlip4 = 0x64086408u;

// Four exact e4m3 bytes (samples in order) from two fp16 pairs whose values are integers in
// -8..7, which e4m3 (3 mantissa bits) holds exactly: the conversion cannot round.
__device__ __forceinline__ uint32_t e4m3x4(uint32_t h01, uint32_t h23) {
    __half2_raw a, b;
    a.x = (unsigned short)(h01 & 0xFFFFu);
    a.y = (unsigned short)(h01 >> 16);
    b.x = (unsigned short)(h23 & 0xFFFFu);
    b.y = (unsigned short)(h23 >> 16);
    const uint32_t lo = __nv_cvt_halfraw2_to_fp8x2(a, __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_halfraw2_to_fp8x2(b, __NV_SATFINITE, __NV_E4M3);
    return (lo & 0xFFFFu) | (hi << 16);
}

}  // namespace conv
}  // namespace corr
