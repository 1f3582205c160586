// Box codecs of the physical layouts, compiled for the host packer and for
// the device refit alike (one implementation, identical IEEE arithmetic on
// both sides: no contraction, correctly rounded double and float ops).
//
// Every encoder writes a box that encloses its input: f32 as is, f16 and
// world-grid codes rounded outward, u8 codes verified against the device
// decode and bumped until they enclose (App. D.2 reading). Inputs are the
// exact boxes; each encoder applies the build pad itself (`padded`).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "layout.h"

namespace scion {

struct Box3 {
  float lo[3], hi[3];
};

// ------------------------------------------------------------ directed rounding
// double -> float toward -inf / +inf
SCION_HD float round_down_f32(double x) {
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, -INFINITY);
  return f;
}
SCION_HD float round_up_f32(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

// Directed rounding of the exact value s + e to float (e is the error term
// of an error-free transform, at most half an ulp of s): the nearest float to
// s is at most one step away from the wanted one, and the comparison with
// s + e decides the step exactly.
SCION_HD float round_dir(double s, double e, int dir) {
  float f = (float)s;
  if (isnan(f)) return f;
  const bool above = (double)f > s || ((double)f == s && e < 0.0);
  const bool below = (double)f < s || ((double)f == s && e > 0.0);
  if (dir < 0 && above) f = nextafterf(f, -INFINITY);
  if (dir > 0 && below) f = nextafterf(f, INFINITY);
  return f;
}
// float products are exact in double (24 + 24 significant bits)
SCION_HD float mul_rd_f32(float a, float b) { return round_dir((double)a * (double)b, 0.0, -1); }
// a + b with Knuth's TwoSum error term, rounded toward dir
SCION_HD float add_dir(double x, double y, int dir) {
  const double s = x + y;
  if (!isfinite(s)) return (float)s;
  const double bb = s - x, e = (x - (s - bb)) + (y - bb);
  return round_dir(s, e, dir);
}
SCION_HD float add_rd_f32(float a, float b) { return add_dir(a, b, -1); }
SCION_HD float sub_rd_f32(float a, float b) { return add_dir(a, -(double)b, -1); }
SCION_HD float sub_ru_f32(float a, float b) { return add_dir(a, -(double)b, +1); }
// largest float f with f * d <= n (n >= 0, d > 0 finite); f * d is exact in double
SCION_HD float div_rd_f32(float n, float d) {
  float f = (float)((double)n / (double)d);
  while (f > 0.0f && (double)f * (double)d > (double)n) f = nextafterf(f, -INFINITY);
  for (int i = 0; i < 4; ++i) {
    const float g = nextafterf(f, INFINITY);
    if (isfinite(g) && (double)g * (double)d <= (double)n) f = g;
    else break;
  }
  return f;
}

// ------------------------------------------------------------ f16
SCION_HD float f16_to_f32(uint16_t h) {
  const uint32_t s = h >> 15, e = (h >> 10) & 31u, m = h & 1023u;
  double v;
  if (e == 0) v = ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp((double)(1024u + m), (int)e - 25);
  return (float)(s ? -v : v);
}

// IEEE binary16 with directed rounding: dir < 0 toward -inf, dir > 0 toward +inf.
SCION_HD uint16_t f16_directed(double x, int dir) {
  if (isnan(x)) return 0x7E00;
  if (x == 0.0) return signbit(x) ? 0x8000 : 0;
  const bool neg = x < 0.0;
  const double a = fabs(x);
  uint16_t mag;  // largest finite f16 magnitude <= a
  if (a >= 65504.0) {
    mag = 0x7BFF;
  } else {
    int e;
    frexp(a, &e);    // a = f * 2^e, f in [0.5, 1)
    const int E = e + 14;  // biased exponent of a normal f16 in [2^(E-15), 2^(E-14))
    if (E >= 1) {
      const double f = floor((ldexp(a, 15 - E) - 1.0) * 1024.0);
      mag = (uint16_t)((E << 10) | (int)f);
    } else {
      mag = (uint16_t)floor(ldexp(a, 24));
    }
  }
  const bool exact = (double)f16_to_f32(mag) == a;
  const bool away = (dir > 0 && !neg) || (dir < 0 && neg);
  if (!exact && away) mag = (uint16_t)(mag + 1u);  // 0x7BFF + 1 = +inf pattern
  return (uint16_t)((neg ? 0x8000u : 0u) | mag);
}
SCION_HD uint16_t f32_to_f16_down(float x) { return f16_directed(x, -1); }
SCION_HD uint16_t f32_to_f16_up(float x) { return f16_directed(x, +1); }

// ------------------------------------------------------------ build pad
// World-space pad: 2^-20 * (largest extent + largest |coordinate|), applied
// outward before any encoding so that the traversal's float slab test (with
// its relative margin) never culls a box whose triangle the intersector hits.
SCION_HD Box3 padded(const Box3 &b) {
  double ext = 0.0, mag = 0.0;
  for (int a = 0; a < 3; ++a) {
    ext = fmax(ext, (double)b.hi[a] - (double)b.lo[a]);
    mag = fmax(mag, fmax(fabs((double)b.lo[a]), fabs((double)b.hi[a])));
  }
  const double pad = ldexp(ext + mag, -20);
  Box3 o;
  for (int a = 0; a < 3; ++a) {
    o.lo[a] = round_down_f32((double)b.lo[a] - pad);
    o.hi[a] = round_up_f32((double)b.hi[a] + pad);
  }
  return o;
}
SCION_HD bool box_is_empty(const Box3 &b) { return !(b.lo[0] <= b.hi[0] && b.lo[1] <= b.hi[1] && b.lo[2] <= b.hi[2]); }

SCION_HD void put_u32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }
SCION_HD void put_f32(uint8_t *p, float v) { memcpy(p, &v, 4); }
SCION_HD void put_u16(uint8_t *p, uint16_t v) { memcpy(p, &v, 2); }
SCION_HD uint32_t get_u32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }
SCION_HD float get_f32(const uint8_t *p) { float v; memcpy(&v, p, 4); return v; }
SCION_HD uint16_t get_u16(const uint8_t *p) { uint16_t v; memcpy(&v, p, 2); return v; }

// ------------------------------------------------------------ world grid (q16, eq10)
// q16: coordinate = fma(code, step, wlo), the device arithmetic.
SCION_HD float q16_decode(uint32_t q, float step, float wlo) { return fmaf((float)q, step, wlo); }
// fma with directed rounding: code * bin is exact in double (10 + 24 bits)
SCION_HD float fma_dir(double p, float c, int dir) { return add_dir(p, (double)c, dir); }
// eq10: lo = rd(code * bin + wlo), hi = ru(whi - code * bin), one rounding each.
SCION_HD float eq10_decode_lo(uint32_t q, float bin, float wlo) { return fma_dir((double)q * (double)bin, wlo, -1); }
SCION_HD float eq10_decode_hi(uint32_t q, float bin, float whi) { return fma_dir(-(double)q * (double)bin, whi, +1); }

// q16 step of one axis: the smallest step (from extent / 65535 up) whose last
// code reaches whi.
SCION_HD float q16_step(float wlo, float whi) {
  const double ext = (double)whi - (double)wlo;
  if (!(ext > 0.0)) return 0.0f;
  float step = round_up_f32(ext / (double)kQ16Max);
  while (q16_decode(kQ16Max, step, wlo) < whi) step = nextafterf(step, INFINITY);
  return step;
}
// eq10 bins of one axis (App. D.1 construct_bins_inverse / construct_bins):
// bins_inv = rd(1023 / ru(whi - wlo)) (1 for an empty extent), bin = rd(1 / bins_inv).
SCION_HD void eq10_bins(float wlo, float whi, float *bin, float *bins_inv) {
  float L = sub_ru_f32(whi, wlo);
  if (!(L > 0.0f)) L = 1.0f;
  *bins_inv = div_rd_f32((float)kEq10Max, L);
  *bin = *bins_inv > 0.0f ? div_rd_f32(1.0f, *bins_inv) : 0.0f;
}
SCION_HD uint32_t clamp_code(double v, uint32_t qmax) {
  if (!(v > 0.0)) return 0;
  if (v >= (double)qmax) return qmax;
  return (uint32_t)v;
}
// Codes of one axis of a box; the decoded interval always encloses [lo, hi]
// (verify-and-bump against the exact device decode). Returns false if not.
SCION_HD bool q16_codes(float lo, float hi, float step, float wlo, uint32_t *qlo, uint32_t *qhi) {
  uint32_t a = 0, b = 0;
  if (step > 0.0f) {
    a = clamp_code(floor(((double)lo - (double)wlo) / (double)step), kQ16Max);
    b = clamp_code(ceil(((double)hi - (double)wlo) / (double)step), kQ16Max);
  }
  while (a > 0 && q16_decode(a, step, wlo) > lo) --a;
  while (b < kQ16Max && q16_decode(b, step, wlo) < hi) ++b;
  *qlo = a;
  *qhi = b;
  return q16_decode(a, step, wlo) <= lo && q16_decode(b, step, wlo) >= hi;
}
// eq10 codes: the App. D.1 quantize_lo / quantize_hi (floor of the directed
// products), then verify-and-bump; hi codes count down from whi.
SCION_HD bool eq10_codes(float lo, float hi, float bin, float bins_inv, float wlo, float whi, uint32_t *qlo,
                         uint32_t *qhi) {
  uint32_t a = clamp_code(floor((double)mul_rd_f32(sub_rd_f32(lo, wlo), bins_inv)), kEq10Max);
  uint32_t b = clamp_code(floor((double)mul_rd_f32(sub_rd_f32(whi, hi), bins_inv)), kEq10Max);
  while (a > 0 && eq10_decode_lo(a, bin, wlo) > lo) --a;
  while (b > 0 && eq10_decode_hi(b, bin, whi) < hi) --b;
  *qlo = a;
  *qhi = b;
  return eq10_decode_lo(a, bin, wlo) <= lo && eq10_decode_hi(b, bin, whi) >= hi;
}

// Grid of the world-grid codecs over the padded root box: q16 frame =
// {wlo.xyz, step.xyz, 0, 0, 0}; eq10 frame = {wlo.xyz, whi.xyz, bin.xyz} and
// bins_inv.xyz (used by the encoder only).
SCION_HD void world_frame(uint32_t prec, const Box3 &root_padded, float *frame, float *bins_inv) {
  for (int a = 0; a < 3; ++a) {
    frame[a] = root_padded.lo[a];
    bins_inv[a] = 0.0f;
    if (prec == PREC_Q16) {
      frame[3 + a] = q16_step(root_padded.lo[a], root_padded.hi[a]);
      frame[6 + a] = 0.0f;
    } else {
      frame[3 + a] = root_padded.hi[a];
      eq10_bins(root_padded.lo[a], root_padded.hi[a], &frame[6 + a], &bins_inv[a]);
    }
  }
}

// ------------------------------------------------------------ own-box node box
// Write the own box (exact, padded here) of an own-box node at p: f32 corners
// (24 B), q16 codes (12 B) or eq10 lo/hi code words (8 B). An empty box is
// written so that no ray enters it (f32) or as the widest codes' inverse
// (codes: lo = top of the grid, hi = bottom). False if a code cannot enclose.
SCION_HD bool encode_own_box(uint32_t prec, const Box3 &exact, const float *frame, const float *bins_inv,
                             uint8_t *p) {
  const bool empty = box_is_empty(exact);
  const Box3 b = empty ? exact : padded(exact);
  if (prec == PREC_F32) {
    for (int a = 0; a < 3; ++a) {
      put_f32(p + 4 * a, empty ? INFINITY : b.lo[a]);
      put_f32(p + 12 + 4 * a, empty ? -INFINITY : b.hi[a]);
    }
    return true;
  }
  bool ok = true;
  uint32_t qlo[3], qhi[3];
  for (int a = 0; a < 3; ++a) {
    if (empty) {
      qlo[a] = prec == PREC_Q16 ? kQ16Max : kEq10Max;
      qhi[a] = prec == PREC_Q16 ? 0u : kEq10Max;
      continue;
    }
    ok &= prec == PREC_Q16 ? q16_codes(b.lo[a], b.hi[a], frame[3 + a], frame[a], &qlo[a], &qhi[a])
                           : eq10_codes(b.lo[a], b.hi[a], frame[6 + a], bins_inv[a], frame[a], frame[3 + a],
                                        &qlo[a], &qhi[a]);
  }
  if (prec == PREC_Q16) {
    for (int a = 0; a < 3; ++a) {
      put_u16(p + 2 * a, (uint16_t)qlo[a]);
      put_u16(p + 6 + 2 * a, (uint16_t)qhi[a]);
    }
  } else {
    put_u32(p, eq10_pack(qlo[0], qlo[1], qlo[2]));
    put_u32(p + 4, eq10_pack(qhi[0], qhi[1], qhi[2]));
  }
  return ok;
}

// ------------------------------------------------------------ shared-slab node
// Split planes of a shared-slab node from its children's exact boxes: the
// left child keeps the node's carried box with hi[axis] = slo, the right one
// with lo[axis] = shi; slo and shi are the padded children's planes, so each
// child's carried box encloses its padded box (the node's carried box already
// encloses the node's padded box, and a child's pad is at most its parent's).
SCION_HD void encode_slab_planes(const Box3 &left_exact, const Box3 &right_exact, uint32_t axis, uint8_t *p) {
  const bool le = box_is_empty(left_exact), re = box_is_empty(right_exact);
  put_f32(p, le ? -INFINITY : padded(left_exact).hi[axis]);
  put_f32(p + 4, re ? INFINITY : padded(right_exact).lo[axis]);
}

// ------------------------------------------------------------ wide node boxes
// u8 / u16 frame decode: coordinate = fma(q, 2^e, origin), the device arithmetic.
SCION_HD float u8_decode(uint32_t q, float scale, float origin) { return fmaf((float)q, scale, origin); }

// Write the W child boxes of a wide node (children 0..n-1 given as exact
// boxes, padded here; slots n..W-1 and empty boxes are written as empty) and,
// for u8 / u16, the node's frame header. Returns 0, or 2 (f16) / 4 (u8, u16) when a code
// could not enclose its box.
SCION_HD int encode_wide_boxes(uint32_t W, uint32_t prec, uint32_t soa, const Box3 *exact, uint32_t n,
                               uint8_t *p) {
  int bad = 0;
  Box3 cb[8];
  bool live[8];
  for (uint32_t k = 0; k < W; ++k) {
    live[k] = k < n && !box_is_empty(exact[k]);
    if (live[k]) cb[k] = padded(exact[k]);
  }
  if (prec == PREC_F32) {
    for (uint32_t k = 0; k < W; ++k)
      for (uint32_t c = 0; c < 6; ++c) {
        const float v = live[k] ? (c < 3 ? cb[k].lo[c] : cb[k].hi[c - 3]) : (c < 3 ? INFINITY : -INFINITY);
        put_f32(p + wide_box_offset(W, prec, soa, k, c), v);
      }
    return 0;
  }
  if (prec == PREC_F16) {
    for (uint32_t k = 0; k < W; ++k)
      for (uint32_t c = 0; c < 6; ++c) {
        uint16_t h;
        if (live[k]) {
          h = c < 3 ? f32_to_f16_down(cb[k].lo[c]) : f32_to_f16_up(cb[k].hi[c - 3]);
          const float dec = f16_to_f32(h);
          const bool ok = c < 3 ? dec <= cb[k].lo[c] : dec >= cb[k].hi[c - 3];
          if (!ok) bad |= 2;
        } else {
          h = c < 3 ? 0x7C00 : 0xFC00;  // +inf / -inf: empty
        }
        put_u16(p + wide_box_offset(W, prec, soa, k, c), h);
      }
    return bad;
  }
  // u8 / u16 codes relative to the merged child box (App. D.2), with a guard
  // band of 2^-20 (|coordinate| + extent) beyond the padded boxes, a
  // power-of-two scale per axis, and verify-and-bump against the device decode.
  const uint32_t qmax = prec == PREC_U8 ? 255u : 65535u;
  double mlo[3], mhi[3];
  for (int a = 0; a < 3; ++a) {
    mlo[a] = INFINITY;
    mhi[a] = -INFINITY;
    for (uint32_t k = 0; k < W; ++k)
      if (live[k]) {
        mlo[a] = fmin(mlo[a], (double)cb[k].lo[a]);
        mhi[a] = fmax(mhi[a], (double)cb[k].hi[a]);
      }
  }
  bool any = false;
  for (uint32_t k = 0; k < W; ++k) any |= live[k];
  if (!any)
    for (int a = 0; a < 3; ++a) mlo[a] = mhi[a] = 0.0;
  double mag = 0.0, ext = 0.0;
  for (int a = 0; a < 3; ++a) {
    mag = fmax(mag, fmax(fabs(mlo[a]), fabs(mhi[a])));
    ext = fmax(ext, mhi[a] - mlo[a]);
  }
  const double g = ldexp(mag + ext, -20);
  float origin[3], scale[3];
  for (int a = 0; a < 3; ++a) {
    origin[a] = round_down_f32(mlo[a] - g);
    const double fhi = (double)round_up_f32(mhi[a] + g);
    const double span = fhi - (double)origin[a];
    int e = -126;
    if (span > 0.0) {
      int ex;
      frexp(span / (double)qmax, &ex);  // span/qmax < 2^ex
      e = ex - 2 > -126 ? ex - 2 : -126;
    }
    while (e < 127 && ldexp((double)qmax, e) < span) ++e;
    scale[a] = (float)ldexp(1.0, e);
    put_f32(p + 4 * a, origin[a]);
    p[12 + a] = (uint8_t)(e + 127);
  }
  for (uint32_t k = 0; k < W; ++k)
    for (int a = 0; a < 3; ++a) {
      uint32_t qlo = qmax, qhi = 0;
      if (live[k]) {
        const double tlo = (double)cb[k].lo[a] - g, thi = (double)cb[k].hi[a] + g;
        const double fl = floor((tlo - origin[a]) / scale[a]);
        const double fh = ceil((thi - origin[a]) / scale[a]);
        qlo = (uint32_t)fmin((double)qmax, fmax(0.0, fl));
        qhi = (uint32_t)fmin((double)qmax, fmax(0.0, fh));
        while (qlo > 0 && (double)u8_decode(qlo, scale[a], origin[a]) > tlo) --qlo;
        while (qhi < qmax && (double)u8_decode(qhi, scale[a], origin[a]) < thi) ++qhi;
        if ((double)u8_decode(qlo, scale[a], origin[a]) > tlo || (double)u8_decode(qhi, scale[a], origin[a]) < thi)
          bad |= 4;
      }
      uint8_t *plo = p + wide_box_offset(W, prec, soa, k, a), *phi = p + wide_box_offset(W, prec, soa, k, 3 + a);
      if (prec == PREC_U8) {
        *plo = (uint8_t)qlo;
        *phi = (uint8_t)qhi;
      } else {
        put_u16(plo, (uint16_t)qlo);
        put_u16(phi, (uint16_t)qhi);
      }
    }
  return bad;
}

}  // namespace scion
