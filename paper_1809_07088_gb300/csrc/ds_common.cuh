// Shared device-side definitions of the GB300 diffuse-scattering library.
//
// Complex arithmetic on float2 / double2, the per-launch parameter blocks, and the error flag
// through which kernels report bounded-wait or argument failures to the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ds {

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using c_t = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ c_t<T> mk(T re, T im) {
    c_t<T> z;
    z.x = re;
    z.y = im;
    return z;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C z;
    z.x = a.x * b.x - a.y * b.y;
    z.y = a.x * b.y + a.y * b.x;
    return z;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) {
    a.y = -a.y;
    return a;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C z;
    z.x = a.x * b.x + a.y * b.y;
    z.y = a.y * b.x - a.x * b.y;
    return z;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) {
    a.x *= s;
    a.y *= s;
    return a;
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C &acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// multiply by i^n
template <typename C> __host__ __device__ __forceinline__ C cipow(C a, int n) {
    C z;
    switch (n & 3) {
    case 0: z = a; break;
    case 1: z.x = -a.y; z.y = a.x; break;
    case 2: z.x = -a.x; z.y = -a.y; break;
    default: z.x = a.y; z.y = -a.x; break;
    }
    return z;
}

// error codes written to the device error word (first writer wins)
enum : int { DEV_OK = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_BOUNDS = 2 };

__device__ __forceinline__ void raise_error(int *flag, int code) {
    if (flag) atomicCAS(flag, 0, code);
}

constexpr int MAX_SITES = 64;     // sites per unit cell handled by the library
constexpr int MAX_FF_CLASSES = 8; // distinct non-constant form factors per request
constexpr double TWO_PI_D = 6.283185307179586476925286766559;
constexpr double FOUR_PI_D = 12.566370614359172953850573533118;

// exponential of the working precision: CUDA's exp in FP64, its fast __expf intrinsic in FP32
// (a few ulp, far inside the FP32 path's error budget)
__device__ __forceinline__ double exp_w(double x) { return exp(x); }
__device__ __forceinline__ float exp_w(float x) { return __expf(x); }
// 2^x: the SFU's approximate base-2 exponential (PTX ex2.approx) in FP32, exp2 in FP64
__device__ __forceinline__ double exp2_w(double x) { return exp2(x); }
__device__ __forceinline__ float exp2_w(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1/x: the SFU's approximate reciprocal (PTX rcp.approx) in FP32, exact division in FP64
// Programmatic dependent launch.  A kernel that ends a producer stage lets the next kernel of its
// stream be scheduled early (launch_dependents: no effect unless that kernel was launched with
// programmatic stream serialization); the consumer runs its independent prologue and then waits
// (griddep_wait) until the preceding grid has completed and its writes are visible.
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// asynchronous global -> shared copies of BYTES (4, 8 or 16) bytes, in commit groups
template <int BYTES> __device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's most recent groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ double rcp_w(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_w(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double div_w(double a, double b) { return a / b; }
__device__ __forceinline__ float div_w(float a, float b) { return __fdividef(a, b); }

// form factor of one class at s^2 = (|Q|/4pi)^2; kind 0 = 1, 1 = 4-Gaussian, 2 = <j0>
template <typename T> __device__ __forceinline__ T form_factor(int kind, const T *c, T s2) {
    if (kind == 1)
        return c[0] * exp_w(-c[4] * s2) + c[1] * exp_w(-c[5] * s2) + c[2] * exp_w(-c[6] * s2) +
               c[3] * exp_w(-c[7] * s2) + c[8];
    if (kind == 2) {
        T f = c[6] + c[0] * exp_w(-c[1] * s2) + c[2] * exp_w(-c[3] * s2);
        if (c[4] != T(0)) f += c[4] * exp_w(-c[5] * s2);
        return f;
    }
    return T(1);
}

} // namespace ds
