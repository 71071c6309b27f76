/*
 * Host restatement, for testing, of the binary32 reconstruction the decode
 * kernels use for codes below 2^23 (Eq. quantization, Q2): the product
 * (2q+1) e split exactly by a fused multiply-add, m + ph split exactly by
 * TwoSum, and RN(m + ph + pl) formed as RN(th + RO(tl + pl)), RO rounding to
 * odd (Boldo and Melquiond, "Emulation of FMA and correctly rounded sums:
 * proved algorithms using rounding to odd", IEEE Trans. Computers 57(4),
 * 2008).  Directed roundings come from fesetround; every intermediate is kept
 * in a volatile float so that no operation moves across a mode change.
 * Returns 0 where the kernels fall back (q out of range, subnormal result).
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

static float add_mode(float a, float b, int mode) {
  fesetround(mode);
  volatile float va = a, vb = b;
  volatile float r = va + vb;
  fesetround(FE_TONEAREST);
  return r;
}

static int q2_ro(int64_t q, float m, float e, float *out) {
  if (q < 0 || q >= (1 << 23)) return 0;
  volatile float qf = (float)(2 * q + 1);
  volatile float ph = qf * e;
  volatile float pl = fmaf(qf, e, -ph);
  volatile float th = m + ph;
  volatile float bb = th - m;
  volatile float aa = th - bb;
  volatile float tl = (m - aa) + (ph - bb);
  float rz = add_mode(tl, pl, FE_TOWARDZERO);
  const int inexact = add_mode(tl, pl, FE_UPWARD) != add_mode(tl, pl, FE_DOWNWARD);
  uint32_t b;
  memcpy(&b, &rz, 4);
  b |= inexact ? 1u : 0u;
  volatile float v;
  memcpy((void *)&v, &b, 4);
  volatile float z = th + v;
  if (z == 0.0f) {
    *out = 0.0f;
    return 1;
  }
  if (fabsf(z) < 0x1p-126f) return 0;
  *out = z;
  return 1;
}

void q2_ro_many(const int64_t *q, size_t n, float m, float e, float *out, int *ok) {
  for (size_t i = 0; i < n; ++i) ok[i] = q2_ro(q[i], m, e, &out[i]);
}
