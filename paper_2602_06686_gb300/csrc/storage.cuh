// storage.cuh -- population storage formats and vectorised plane access.
//
// Every format stores the shifted population df_i = f_i - w_i rho0, so that the
// stored magnitudes are the (small) deviations from the rest state: FP64 and
// FP32 keep more significant digits of the flow signal, and FP16/BF16 become
// usable at all.  Encoding rounds to nearest even; FP16 keeps subnormals.
// Arithmetic type R is double for FP64 storage and float otherwise.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cstring>

namespace lbm {

struct StF64 {
  using T = double;
  using R = double;
  static constexpr int id = 0;
  static constexpr int VBYTES = 16;
  __device__ __forceinline__ static R dec(T v) { return v; }
  __device__ __forceinline__ static T enc(R v) { return v; }
};
struct StF32 {
  using T = float;
  using R = float;
  static constexpr int id = 1;
  static constexpr int VBYTES = 16;
  __device__ __forceinline__ static R dec(T v) { return v; }
  __device__ __forceinline__ static T enc(R v) { return v; }
};
struct StF16 {
  using T = __half;
  using R = float;
  static constexpr int id = 2;
  static constexpr int VBYTES = 16;
  __device__ __forceinline__ static R dec(T v) { return __half2float(v); }
  __device__ __forceinline__ static T enc(R v) { return __float2half_rn(v); }
  // two adjacent elements as one 32-bit word (element a in the low half)
  __device__ __forceinline__ static void dec2(uint32_t w, R& a, R& b) {
    __half2 h;
    memcpy(&h, &w, 4);
    const float2 f = __half22float2(h);
    a = f.x;
    b = f.y;
  }
  __device__ __forceinline__ static uint32_t enc2(R a, R b) {
    const __half2 h = __floats2half2_rn(a, b);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
  }
};
struct StBF16 {
  using T = __nv_bfloat16;
  using R = float;
  static constexpr int id = 3;
  static constexpr int VBYTES = 16;
  __device__ __forceinline__ static R dec(T v) { return __bfloat162float(v); }
  __device__ __forceinline__ static T enc(R v) { return __float2bfloat16_rn(v); }
  __device__ __forceinline__ static void dec2(uint32_t w, R& a, R& b) {
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    const float2 f = __bfloat1622float2(h);
    a = f.x;
    b = f.y;
  }
  __device__ __forceinline__ static uint32_t enc2(R a, R b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
  }
};

template <int BYTES>
struct RawT;
template <>
struct RawT<1> {
  using type = unsigned char;
};
template <>
struct RawT<2> {
  using type = unsigned short;
};
template <>
struct RawT<4> {
  using type = unsigned int;
};
template <>
struct RawT<8> {
  using type = uint2;
};
template <>
struct RawT<16> {
  using type = uint4;
};

// Load policies: LD_NC reads through the non-coherent (texture / L1) path, valid
// when the buffer was written by an earlier kernel launch; LD_CG caches in L2
// only, required when another SM of the SAME launch wrote the data (the
// persistent batched kernel), since L1 is not coherent across SMs.
enum { LD_NC = 0, LD_CG = 1 };

template <int LD>
__device__ __forceinline__ unsigned char ld_raw(const unsigned char* p) {
  return LD == LD_CG ? __ldcg(p) : __ldg(p);
}
template <int LD>
__device__ __forceinline__ unsigned short ld_raw(const unsigned short* p) {
  return LD == LD_CG ? __ldcg(p) : __ldg(p);
}
template <int LD>
__device__ __forceinline__ unsigned int ld_raw(const unsigned int* p) {
  return LD == LD_CG ? __ldcg(p) : __ldg(p);
}
template <int LD>
__device__ __forceinline__ uint2 ld_raw(const uint2* p) {
  return LD == LD_CG ? __ldcg(p) : __ldg(p);
}
template <int LD>
__device__ __forceinline__ uint4 ld_raw(const uint4* p) {
  return LD == LD_CG ? __ldcg(p) : __ldg(p);
}

// NV consecutive elements starting at p (p aligned to NV * sizeof(T)).
template <typename T, int NV, int LD = LD_NC>
__device__ __forceinline__ void ld_vec(const T* p, T (&out)[NV]) {
  using Raw = typename RawT<sizeof(T) * NV>::type;
  Raw r = ld_raw<LD>(reinterpret_cast<const Raw*>(p));
  memcpy(out, &r, sizeof(Raw));
}

template <class S, int NV, int LD = LD_NC>
__device__ __forceinline__ void ld_dec(const typename S::T* p, typename S::R (&out)[NV]) {
  typename S::T t[NV];
  ld_vec<typename S::T, NV, LD>(p, t);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = S::dec(t[k]);
}

// One element.
template <class S, int LD = LD_NC>
__device__ __forceinline__ typename S::R ld1(const typename S::T* p) {
  typename S::T t[1];
  ld_vec<typename S::T, 1, LD>(p, t);
  return S::dec(t[0]);
}

template <class S, int NV>
__device__ __forceinline__ void st_enc(typename S::T* p, const typename S::R (&v)[NV]) {
  using Raw = typename RawT<sizeof(typename S::T) * NV>::type;
  typename S::T t[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) t[k] = S::enc(v[k]);
  Raw r;
  memcpy(&r, t, sizeof(Raw));
  *reinterpret_cast<Raw*>(p) = r;
}

}  // namespace lbm
