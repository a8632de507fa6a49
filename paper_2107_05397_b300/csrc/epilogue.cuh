// Output epilogue shared by the pair kernels: placement of one distance in the
// caller's buffer for the three layouts of the C ABI (full, condensed, stripes).
#pragma once

#include "ufb_internal.cuh"

namespace ufb {

// V = float (mixed-precision kernels, FP32 outputs) or double (FP64 kernels);
// a value is converted only when its type differs from the output's.
template <typename V>
__device__ __forceinline__ void put_value(const OutSpec &o, int64_t idx, V d) {
  if (o.is_f64)
    static_cast<double *>(o.out)[idx] = static_cast<double>(d);
  else
    static_cast<float *>(o.out)[idx] = static_cast<float>(d);
}

// Distance from the two sums of the pair.  A zero denominator (both samples
// empty, only zero-length branches) gives 0; results are clamped to [0, 1],
// the range of the definition, to absorb last-bit rounding.
__device__ __forceinline__ double ratio01(double num, double den) {
  if (!(den > 0.0)) return 0.0;
  double d = num / den;
  return fmin(1.0, fmax(0.0, d));
}

// Mixed-precision form: the two sums are exact (or FP64) and only the final
// ratio is taken in FP32, the precision of the output (relative error of the
// quotient below 2^-22, so at most ~3e-7 absolute on a value in [0, 1]).
__device__ __forceinline__ float ratio01_f32(float num, float den) {
  if (!(den > 0.f)) return 0.f;
  const float d = __fdiv_rn(num, den);
  return fminf(1.f, fmaxf(0.f, d));
}

// Writes d(li, lj) for local sample indices li < lj of study `st`.
//   stripe form: stripe s, element k holds d(k, (k+s+1) mod n); the pair is
//   element li of stripe lj-li-1 and element lj of stripe n-(lj-li)-1, each
//   when that stripe exists (s < ceil((n-1)/2)) and lies in [s0, s1).
//   condensed / full: written when its stripe min(lj-li-1, n-(lj-li)-1) is in
//   [s0, s1).
template <typename V>
__device__ __forceinline__ void put_pair(const OutSpec &o, const StudyDev &st, int li,
                                         int lj, V d) {
  const int n = st.n;
  const int delta = lj - li;
  const int sa = delta - 1;
  const int sb = n - delta - 1;
  const int nst = n >> 1;  // ceil((n-1)/2)
  if (o.layout == UNIFRAC_OUT_STRIPES) {
    if (sa >= o.s0 && sa < o.s1 && sa < nst)
      put_value(o, st.out_off + (int64_t)(sa - o.s0) * n + li, d);
    if (sb >= o.s0 && sb < o.s1 && sb < nst)
      put_value(o, st.out_off + (int64_t)(sb - o.s0) * n + lj, d);
    return;
  }
  const int s = sa < sb ? sa : sb;
  if (s < o.s0 || s >= o.s1) return;
  if (o.layout == UNIFRAC_OUT_CONDENSED) {
    const int64_t idx = (int64_t)li * n - (int64_t)li * (li + 1) / 2 + (lj - li - 1);
    put_value(o, st.out_off + idx, d);
  } else {
    put_value(o, st.out_off + (int64_t)li * n + lj, d);
    put_value(o, st.out_off + (int64_t)lj * n + li, d);
  }
}

// Full layout only: the zero diagonal, written by the diagonal tiles.
__device__ __forceinline__ void put_diag(const OutSpec &o, const StudyDev &st, int li) {
  if (o.layout == UNIFRAC_OUT_FULL) put_value(o, st.out_off + (int64_t)li * st.n + li, 0.f);
}

}  // namespace ufb
