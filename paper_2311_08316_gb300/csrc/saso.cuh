// SASO sketching operator S (d x m) of Sec. 2.3.1: column r holds exactly s
// nonzeros at distinct, uniformly chosen rows, each +-1/sqrt(s) with equal
// probability.  Columns are generated on the device from (seed, r) with the
// counter-based Philox4x32-10 generator (Salmon et al., SC'11), so S is never
// stored densely and any column can be regenerated independently.
//
// Library reading (identical on every caller of this header):
//   key = (seed lo, seed hi); row draws read the words of
//   Philox(ctr = (r lo, r hi, t, 0)) for t = 0, 1, ...; sign draws read
//   Philox(ctr = (r lo, r hi, t, 1)).  Rows: Floyd's algorithm (for q-th
//   draw, range [0, d-s+q]; a repeat takes d-s+q instead), each uniform draw
//   by Lemire's multiply-shift with at most 64 rejections.  Nonzero q is
//   negative iff bit q mod 32 of sign word q/32 is set.
#pragma once
#include <cstdint>

namespace cqrrpt {

struct Philox4 {
  uint32_t v[4];
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t a = (uint64_t)0xD2511F53u * c0;
    const uint64_t b = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t x0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
    const uint32_t x2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)b;
    c3 = (uint32_t)a;
    c0 = x0;
    c2 = x2;
  }
  Philox4 out;
  out.v[0] = c0; out.v[1] = c1; out.v[2] = c2; out.v[3] = c3;
  return out;
}

// Sequential word reader over one Philox stream of column r.
struct PhiloxWords {
  uint32_t k0, k1, r0, r1, tag, block;
  Philox4 buf;
  int pos;
  __host__ __device__ __forceinline__ PhiloxWords(uint64_t seed, int64_t r, uint32_t t)
      : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), r0((uint32_t)(uint64_t)r),
        r1((uint32_t)((uint64_t)r >> 32)), tag(t), block(0), pos(4) {}
  __host__ __device__ __forceinline__ uint32_t next() {
    if (pos == 4) {
      buf = philox4x32_10(r0, r1, block, tag, k0, k1);
      ++block;
      pos = 0;
    }
    return buf.v[pos++];
  }
};

__host__ __device__ __forceinline__ uint32_t lemire_below(PhiloxWords& w, uint32_t range) {
  uint64_t prod = (uint64_t)w.next() * range;
  uint32_t low = (uint32_t)prod;
  if (low < range) {
    const uint32_t thresh = (0u - range) % range;
    for (int tries = 0; low < thresh && tries < 64; ++tries) {
      prod = (uint64_t)w.next() * range;
      low = (uint32_t)prod;
    }
  }
  return (uint32_t)(prod >> 32);
}

// Writes the s rows (draw order) of column r to rows[0..s) and the negative
// flags as bits of *negbits (bit q = nonzero q); s <= kMaxNnzInline.
constexpr int kMaxNnzInline = 32;

__host__ __device__ __forceinline__ void saso_column(uint64_t seed, int64_t r, int d, int s,
                                                     int* rows, uint32_t* negbits) {
  PhiloxWords rw(seed, r, 0u);
  for (int q = 0; q < s; ++q) {
    const uint32_t top = (uint32_t)(d - s + q);
    const uint32_t t = lemire_below(rw, top + 1u);
    bool taken = false;
    for (int p = 0; p < q; ++p) taken |= ((uint32_t)rows[p] == t);
    rows[q] = (int)(taken ? top : t);
  }
  PhiloxWords sw(seed, r, 1u);
  *negbits = sw.next();
}

}  // namespace cqrrpt
