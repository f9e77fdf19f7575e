// amr_internal.cuh -- device-side building blocks shared by the index and
// hydro kernels of the GB300 level-advance library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "amr.h"

namespace amr {

constexpr int kMaxLev = 15;
constexpr int kNV = 5;
constexpr uint64_t kEmpty = ~0ull;     // empty hash slot
constexpr int32_t kPending = 0x7FFFFFFF;  // claimed ghost key, slot not final

// device error word bits
enum : int {
  kErrGrading = 1,
  kErrDup = 2,
  kErrTableFull = 4,
  kErrNaN = 8,
  kErrRange = 16,
  kErrClaimOverflow = 32,
  kErrCacheMismatch = 64,
  kErrTimeout = 128,
  kErrIndex = 256,  // bounds-checked builds: an index-table entry out of range
};

// Bounds-checked builds (compiled with AMR_CHECKED): an index read from an
// index table is tested against the extent of what it addresses; a bad one
// sets kErrIndex in the error word and is replaced by `fallback`, so that no
// access leaves its array.  Plain builds pass the index through.
#ifdef AMR_CHECKED
__device__ __forceinline__ int64_t checked(int64_t i, int64_t lo, int64_t hi, int *err,
                                           int64_t fallback = 0) {
  if (i < lo || i >= hi) {
    atomicOr(err, kErrIndex);
    return fallback;
  }
  return i;
}
#else
__device__ __forceinline__ int64_t checked(int64_t i, int64_t, int64_t, int *, int64_t = 0) {
  return i;
}
#endif

// ---------------------------------------------------------------------------
// keys (Sec. 2.1).  External keys (the C ABI's): level in bits 60..63, i/j/k
// in three 20-bit fields.  Internal keys also carry the member mesh of a
// batched handle: member in bits 49..63, level in 45..48, i/j/k in three
// 15-bit fields (levels <= 15 keep coordinates below 2^14).
// ---------------------------------------------------------------------------
constexpr int kMaxMembers = 1 << 15;

__host__ __device__ __forceinline__ uint64_t key_pack(int l, uint32_t i, uint32_t j, uint32_t k) {
  return (uint64_t(l) << 60) | (uint64_t(i) << 40) | (uint64_t(j) << 20) | uint64_t(k);
}
__host__ __device__ __forceinline__ uint64_t ikey(int m, int l, uint32_t i, uint32_t j, uint32_t k) {
  return (uint64_t(m) << 49) | (uint64_t(l) << 45) | (uint64_t(i) << 30) | (uint64_t(j) << 15) |
         uint64_t(k);
}
__host__ __device__ __forceinline__ int ikey_member(uint64_t key) { return int(key >> 49); }
__host__ __device__ __forceinline__ int ikey_lev(uint64_t key) { return int(key >> 45) & 15; }
__host__ __device__ __forceinline__ uint32_t ikey_x(uint64_t key) { return uint32_t(key >> 30) & 0x7FFFu; }
__host__ __device__ __forceinline__ uint32_t ikey_y(uint64_t key) { return uint32_t(key >> 15) & 0x7FFFu; }
__host__ __device__ __forceinline__ uint32_t ikey_z(uint64_t key) { return uint32_t(key) & 0x7FFFu; }
// same member and coordinates, another level
__host__ __device__ __forceinline__ uint64_t ikey_at(uint64_t key, int l, uint32_t i, uint32_t j,
                                                    uint32_t k) {
  return ikey(ikey_member(key), l, i, j, k);
}
__host__ __device__ __forceinline__ uint64_t external_key(uint64_t key) {
  return key_pack(ikey_lev(key), ikey_x(key), ikey_y(key), ikey_z(key));
}

// FNV-1a 64 over the key's 8 bytes, least significant byte first (Sec. 6).
__device__ __forceinline__ uint64_t fnv1a64(uint64_t key) {
  uint64_t h = 0xcbf29ce484222325ull;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    h ^= (key >> (8 * b)) & 0xFFull;
    h *= 0x100000001b3ull;
  }
  return h;
}

// Lanes of the warp with the same digit as this lane (nbits <= 8; radix-sort digits), from one
// ballot per digit bit: cheaper on this GPU than __match_any_sync.  Invalid
// lanes (past the end) match only each other.
__device__ __forceinline__ unsigned digit_peers(unsigned dig, int nbits, bool valid) {
  const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
  unsigned peers = valid ? vm : ~vm;
  for (int b = 0; b < nbits; ++b) {
    const bool bit = (dig >> b) & 1u;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, bit);
    peers &= bit ? m : ~m;
  }
  return peers;
}

// 3-D Hilbert index with `bits` bits per axis, x the most significant axis
// (Skilling's transposed-coordinate construction, AIP Conf. Proc. 707, 2004).
__device__ __forceinline__ uint64_t hilbert_index(uint32_t x, uint32_t y, uint32_t z, int bits) {
  if (bits <= 0) return 0;
  uint32_t a0 = x, a1 = y, a2 = z;
  for (int b = bits - 1; b >= 1; --b) {
    const uint32_t q = 1u << b, m = q - 1u;
    // axis 0
    if (a0 & q) a0 ^= m;
    // axis 1
    if (a1 & q) {
      a0 ^= m;
    } else {
      const uint32_t t = (a0 ^ a1) & m;
      a0 ^= t;
      a1 ^= t;
    }
    // axis 2
    if (a2 & q) {
      a0 ^= m;
    } else {
      const uint32_t t = (a0 ^ a2) & m;
      a0 ^= t;
      a2 ^= t;
    }
  }
  a1 ^= a0;
  a2 ^= a1;
  uint32_t g = 0;
  for (int b = bits - 1; b >= 1; --b)
    if (a2 & (1u << b)) g ^= (1u << b) - 1u;
  a0 ^= g;
  a1 ^= g;
  a2 ^= g;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b) {
    h = (h << 3) | (uint64_t((a0 >> b) & 1u) << 2) | (uint64_t((a1 >> b) & 1u) << 1) |
        uint64_t((a2 >> b) & 1u);
  }
  return h;
}

// ---------------------------------------------------------------------------
// hash table: open addressing, linear probing, keys u64 (kEmpty = free),
// values i32 = 1-based oct index (0 = tombstone / not found).
// ---------------------------------------------------------------------------
struct HashView {
  uint64_t *key;
  int32_t *val;
  uint64_t mask;  // capacity - 1 (capacity a power of two)
};

// Insert or find `key`; returns the slot and whether this call inserted it.
__device__ __forceinline__ uint64_t hash_insert(HashView h, uint64_t key, bool *inserted, int *err) {
  uint64_t s = fnv1a64(key) & h.mask;
  for (uint64_t n = 0; n <= h.mask; ++n) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long *>(h.key + s), (unsigned long long)kEmpty,
                  (unsigned long long)key);
    if (prev == kEmpty) {
      *inserted = true;
      return s;
    }
    if (prev == key) {
      *inserted = false;
      return s;
    }
    s = (s + 1) & h.mask;
  }
  atomicOr(err, kErrTableFull);
  *inserted = false;
  return ~0ull;
}

// Cooperative lookup by the 8 lanes of an aligned lane group, all holding
// the same key: each round reads 8 consecutive slots (one 64-byte run) and
// decides with one ballot.  Returns the stored value (0 if absent) in every
// lane of the group.  Linear probing never leaves an empty slot between a
// key's home slot and the key, so the first empty slot ends the search.
__device__ __forceinline__ int32_t hash_probe8(HashView h, uint64_t key) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned base = lane & ~7u;
  const unsigned gmask = 0xFFu << base;
  const unsigned sub = lane & 7u;
  const uint64_t home = fnv1a64(key) & h.mask;
  for (uint64_t r = 0; r <= h.mask; r += 8) {
    const uint64_t s = (home + r + sub) & h.mask;
    const uint64_t k = __ldcg(reinterpret_cast<const unsigned long long *>(h.key + s));
    const unsigned hit = __ballot_sync(gmask, k == key) & gmask;
    const unsigned emp = __ballot_sync(gmask, k == kEmpty) & gmask;
    const unsigned hit_first = hit ? __ffs(hit) - 1 : 32u;
    const unsigned emp_first = emp ? __ffs(emp) - 1 : 32u;
    if (hit && hit_first < emp_first) {
      int32_t v = (lane == hit_first) ? __ldcg(h.val + s) : 0;
      return __shfl_sync(gmask, v, int(hit_first));
    }
    if (emp) return 0;
  }
  return 0;
}

// Single-thread lookup (for sparse use inside other kernels).
__device__ __forceinline__ int32_t hash_probe1(HashView h, uint64_t key) {
  uint64_t s = fnv1a64(key) & h.mask;
  for (uint64_t n = 0; n <= h.mask; ++n) {
    const uint64_t k = __ldcg(reinterpret_cast<const unsigned long long *>(h.key + s));
    if (k == key) return __ldcg(h.val + s);
    if (k == kEmpty) return 0;
    s = (s + 1) & h.mask;
  }
  return 0;
}

// x modulo a power-of-two period (cells or octs per axis of a level)
__device__ __forceinline__ uint32_t wrapc(int64_t x, int64_t period) {
  return uint32_t(x & (period - 1));
}

// Face directions: 2d = minus side, 2d+1 = plus side, d = 0 (x), 1 (y), 2 (z).
// Index of the face neighbour in the 27-neighbour array ((dz,dy,dx) order).
__host__ __device__ __forceinline__ int face_to_nbr27(int f) {
  const int d = f >> 1, s = (f & 1) ? 1 : -1;
  return 13 + s * (d == 0 ? 1 : (d == 1 ? 3 : 9));
}

}  // namespace amr
