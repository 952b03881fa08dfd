// 16-bit deviation storage of the populations (precisions LBM_FP16_DEV and
// LBM_BF16_DEV): element tag and conversions.  Not part of the C ABI.
//
// Per node and component the state holds rho* (the post-collision density,
// float32), f*_0 (float32) and, for i = 1..18, the 16-bit deviation
//     d_i(x) = f*_i(x) - w_i rho(x + c_i)
// of the moving population from the equilibrium weight of the density of the
// node it streams to.  The writer holds rho(x + c_i) in its on-chip density
// planes (the force of Eq. 7 needs the same 18 neighbour densities), and the
// reader y = x + c_i rebuilds the pulled value as w_i rho*(y) + d_i(x) from
// its own rho*, so no neighbour density is read from memory.  The rest
// population is stored as the remainder f*_0 = rho - sum_i (w_i rho(x + c_i)
// + d_i), which makes the rebuilt populations of a node sum to its density:
// mass is conserved to float32 rounding whatever the 16-bit rounding.
// Populations that leave the box are rebuilt with the ghost density.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmgb {
namespace {

// One 16-bit unit of the deviation layout; T = __half or __nv_bfloat16
// names the format of the deviations.
template <typename T>
struct Dev {
    unsigned short bits;
};

template <typename S>
struct is_dev_t {
    static constexpr bool value = false;
};
template <typename T>
struct is_dev_t<Dev<T>> {
    static constexpr bool value = true;
};

// The deviation format of a Dev<T> storage tag (declaration only, for decltype).
template <typename T>
T dev_tag(Dev<T>);

template <typename T>
__device__ __forceinline__ float dev_to_f(unsigned short b);
template <>
__device__ __forceinline__ float dev_to_f<__half>(unsigned short b) {
    return __half2float(__ushort_as_half(b));
}
template <>
__device__ __forceinline__ float dev_to_f<__nv_bfloat16>(unsigned short b) {
    // bfloat16 is the upper half of a float32
    return __uint_as_float((unsigned)b << 16);
}

// Round to nearest even.
template <typename T>
__device__ __forceinline__ unsigned short dev_from_f(float v);
template <>
__device__ __forceinline__ unsigned short dev_from_f<__half>(float v) {
    return __half_as_ushort(__float2half_rn(v));
}
template <>
__device__ __forceinline__ unsigned short dev_from_f<__nv_bfloat16>(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// The two deviations {A, B} of one direction and node share a 32-bit word
// (A in the low half).
template <typename T>
__device__ __forceinline__ float2 dev_unpack2(unsigned w);
template <>
__device__ __forceinline__ float2 dev_unpack2<__half>(unsigned w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}
template <>
__device__ __forceinline__ float2 dev_unpack2<__nv_bfloat16>(unsigned w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// Round a and b to nearest even and pack them (a in the low half).
template <typename T>
__device__ __forceinline__ unsigned dev_pack2(float a, float b);
template <>
__device__ __forceinline__ unsigned dev_pack2<__half>(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}
template <>
__device__ __forceinline__ unsigned dev_pack2<__nv_bfloat16>(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}

}  // namespace
}  // namespace lbmgb
