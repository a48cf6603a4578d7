// Amplitude arithmetic of the two state precisions (device code, shared by
// the sweeps and the H-apply).
//
// FP64 state: a double2 slot is the (re, im) of a complex amplitude.
//
// FP32 state: the amplitudes of this method are real.  The integrals are
// real, the generators tau - tau+ (Eq. 4) are real matrices in the
// occupation basis and the reference determinant is real, so every state
// of the ansatz (Eq. 3 / Eq. 5) and every H psi (Eq. 2) is real.  A float2
// slot therefore holds ONE real amplitude as the unevaluated sum hi + lo of
// two FP32 words: hi is the amplitude rounded to FP32, lo the rounding error
// that the kernels restore with error-free transformations (Knuth's TwoSum,
// and FMA for the rounding error of a product).  A rotation rounds each
// amplitude it touches, and every first-order factor touches the reference
// amplitude (about 1) while the adjoint carries H psi components of a few
// Hartree through all factors; in a single FP32 word those roundings
// accumulate to ~1e-6 relative over the 2478 factors of 26 qubits.  With the
// error kept in lo the accumulated error is the rounding of the small
// update terms alone (relative 2^-24 of s*y), about 30 times smaller at 18
// qubits.  Linear maps act on both words alike (H psi, the Trotter-free
// Taylor steps), so their results are again unevaluated sums; only products
// of two amplitudes (energies, norms, gradient dots) need the value hi + lo.
#pragma once
#include <cuda_runtime.h>

namespace uccsd {
namespace amp {

// s + e = a + b exactly, s = fl(a + b) (Knuth's TwoSum; no ordering of |a|,
// |b| needed).  The explicit round-to-nearest intrinsics keep the compiler
// from contracting or reassociating the steps.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Value of an amplitude (FP32: hi + lo; FP64: the real part) in FP64.
__device__ __forceinline__ double value(float2 v) { return (double)v.x + (double)v.y; }

// Re(conj(a) b) in FP64: the product of the two real values for the FP32
// state, the complex form for the FP64 state.
__device__ __forceinline__ double re_dot(float2 a, float2 b) { return value(a) * value(b); }
__device__ __forceinline__ double re_dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

}  // namespace amp
}  // namespace uccsd
