// index_kernels.cuh -- create-time and re-index kernels: oct ordering (level
// bucket sort with prefix sums after a Hilbert-key LSD radix sort, Sec. 2.2),
// the FNV-1a 64 linear-probing hash table (Sec. 2.1, Sec. 6), father/son
// flags, the 27-entry neighbour array and the ghost-oct cache (Sec. 2.3).
// Every oct carries the member mesh it belongs to (a handle may hold many
// independent meshes); neighbours, fathers and ghosts never cross members.
#pragma once
#include "amr_internal.cuh"
#include "scan_kernels.cuh"

namespace amr {

// ---------------------------------------------------------------------------
// input validation and sort keys: (member, level, Hilbert key within level)
// ---------------------------------------------------------------------------
constexpr int kHilbertBits = 42;  // 3 x 14 bits: levels up to 15

__global__ void k_make_sort_keys(const uint8_t *__restrict__ lvl, const uint32_t *__restrict__ ci,
                                 const uint32_t *__restrict__ cj, const uint32_t *__restrict__ ck,
                                 const uint16_t *__restrict__ mem, const uint64_t *__restrict__ hkey_in,
                                 int64_t n, const int *__restrict__ mlmin,
                                 const int *__restrict__ mlmax, uint64_t *__restrict__ comp,
                                 uint32_t *__restrict__ perm, int *__restrict__ err) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const int l = lvl[t];
  const int m = mem[t];
  uint64_t h = 0;
  if (l < mlmin[m] || l > mlmax[m]) {
    atomicOr(err, kErrRange);
  } else {
    const uint32_t side = 1u << (l - 1);
    if (ci[t] >= side || cj[t] >= side || ck[t] >= side) atomicOr(err, kErrRange);
    h = hkey_in ? hkey_in[t] : hilbert_index(ci[t], cj[t], ck[t], l - 1);
    if (h >> kHilbertBits) atomicOr(err, kErrRange);
  }
  comp[t] = (uint64_t(m) << (kHilbertBits + 4)) | (uint64_t(l & 15) << kHilbertBits) |
            (h & ((1ull << kHilbertBits) - 1));
  perm[t] = uint32_t(t);
}

// ---------------------------------------------------------------------------
// a regrid's new oct list: the kept octs in their old (sorted) order, then the
// new octs; the new ones are put in order (below) and the two runs merged by
// rank instead of radix-sorting the whole list (same order: the keys are
// unique)
// ---------------------------------------------------------------------------

// a regrid's new octs in the order the emit pass wrote them: by old oct
// (which is the sorted order of their fathers), then by cell of the father.
// The Hilbert index of an oct is its father's index followed by one octal
// digit, so the list is sorted once each father's group (at most 8 entries,
// at [pos[N + o], pos[N + o + 1]) for old oct o) is sorted; one thread per
// old oct, insertion sort of its group by key
__global__ void k_sort_groups(const uint32_t *__restrict__ pos, int64_t N, uint64_t *__restrict__ key,
                              uint32_t *__restrict__ val) {
  const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (o >= N) return;
  const int64_t a = pos[N + o], b = pos[N + o + 1];
  if (b - a < 2) return;
  uint64_t k[8];
  uint32_t v[8];
  const int m = int(b - a);  // <= 8: one new oct per flagged leaf cell
  for (int t = 0; t < m; ++t) {
    uint64_t kt = key[a + t];
    uint32_t vt = val[a + t];
    int u = t;
    for (; u > 0 && k[u - 1] > kt; --u) {
      k[u] = k[u - 1];
      v[u] = v[u - 1];
    }
    k[u] = kt;
    v[u] = vt;
  }
  for (int t = 0; t < m; ++t) {
    key[a + t] = k[t];
    val[a + t] = v[t];
  }
}

// number of keys of the sorted a[0..n) below x
__device__ __forceinline__ int64_t count_below(const uint64_t *__restrict__ a, int64_t n, uint64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// place every item of the sorted run a (na items) at its rank in the merge
// with the sorted run b (nb items)
__global__ void k_merge_rank(const uint64_t *__restrict__ ak, const uint32_t *__restrict__ av, int64_t na,
                             const uint64_t *__restrict__ bk, int64_t nb, uint64_t *__restrict__ ok,
                             uint32_t *__restrict__ ov) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= na) return;
  const uint64_t k = ak[i];
  const int64_t r = i + count_below(bk, nb, k);
  ok[r] = k;
  ov[r] = av[i];
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (u64 key, u32 value) pairs, one item per thread,
// 256-item tiles: tile histograms -> exclusive scan (digit-major) -> scatter
// with warp-level ranks (one ballot per digit bit) and a warp-ordered prefix.
// ---------------------------------------------------------------------------
constexpr int kRadixTile = 256;
constexpr int kTile = kRadixTile;

// counter[key] += 1 for every calling lane, one atomic per distinct key in
// the warp (sorted inputs give one key per warp: per-lane global atomics on a
// handful of counters serialised at the memory system; shared-memory
// histograms keep per-lane atomics, which are faster there than the match)
__device__ __forceinline__ void warp_count(uint32_t *counter, int key) {
  const unsigned peers = __match_any_sync(__activemask(), key);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(counter + key, uint32_t(__popc(peers)));
}

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int nbits,
                             uint32_t *__restrict__ table, int64_t ntiles) {
  __shared__ uint32_t hist[256];
  const int ndig = 1 << nbits;
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  const int64_t t = blockIdx.x * int64_t(kTile) + threadIdx.x;
  if (t < n) atomicAdd(&hist[(keys[t] >> shift) & uint64_t(ndig - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) table[int64_t(d) * ntiles + blockIdx.x] = hist[d];
}

__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                int shift, int nbits, const uint32_t *__restrict__ offs,
                                int64_t ntiles) {
  __shared__ uint32_t wcnt[kTile / 32][256];
  const int ndig = 1 << nbits;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < (kTile / 32) * 256; q += blockDim.x) (&wcnt[0][0])[q] = 0;
  __syncthreads();
  const int64_t t = blockIdx.x * int64_t(kTile) + threadIdx.x;
  const bool valid = t < n;
  const uint64_t k = valid ? kin[t] : 0;
  const uint32_t v = valid ? vin[t] : 0;
  const unsigned dig = valid ? unsigned((k >> shift) & uint64_t(ndig - 1)) : 0xFFFFFFFFu;
  const unsigned peers = digit_peers(dig, nbits, valid);
  const unsigned rank = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < kTile / 32; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    const uint32_t dst = offs[int64_t(dig) * ntiles + blockIdx.x] + wcnt[warp][dig] + rank;
    kout[dst] = k;
    vout[dst] = v;
  }
}

// ---------------------------------------------------------------------------
// gather octs and state into mesh order; counts octs per (member, level)
// ---------------------------------------------------------------------------
__global__ void k_gather_octs(const uint32_t *__restrict__ perm, const uint8_t *__restrict__ lvl,
                              const uint32_t *__restrict__ ci, const uint32_t *__restrict__ cj,
                              const uint32_t *__restrict__ ck, const uint16_t *__restrict__ mem,
                              int64_t n, uint64_t *__restrict__ key, uint32_t *__restrict__ seg_count) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const uint32_t s = perm[t];
  key[t] = ikey(mem[s], lvl[s], ci[s], cj[s], ck[s]);
  if (seg_count) warp_count(seg_count, 16 * int(mem[s]) + lvl[s]);
}

// the state into mesh order, one thread per cell (the 8 cells of an oct in
// consecutive lanes): oct t of the sorted list takes source oct
// src[perm[t]] (or perm[t] when src is null) of Uin, whose variable v of
// cell 8 q + c sits at v * Sin + 8 q + c; a source of ~0 (a new oct) is left
// as it is (zero)
template <class Tin, class T>
__global__ void k_gather_cells(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ src,
                               const Tin *__restrict__ Uin, int64_t Sin, int64_t n, T *__restrict__ U,
                               int64_t S) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= 8 * n) return;
  const uint32_t s = perm[g >> 3];
  const uint32_t q = src ? src[s] : s;
  if (q == ~0u) return;
  const int64_t from = 8 * int64_t(q) + (g & 7);
#pragma unroll
  for (int v = 0; v < kNV; ++v) U[v * S + g] = T(Uin[v * Sin + from]);
}

// ---------------------------------------------------------------------------
// hash table build, father/son, grading
// ---------------------------------------------------------------------------
__global__ void k_hash_insert(HashView h, const uint64_t *__restrict__ key, int64_t n, int *err) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  bool ins = false;
  const uint64_t s = hash_insert(h, key[t], &ins, err);
  if (s == ~0ull) return;
  if (!ins) {
    atomicOr(err, kErrDup);
    return;
  }
  h.val[s] = int32_t(t + 1);
}

__global__ void k_father_son(HashView h, const uint64_t *__restrict__ key, int64_t n,
                             const int *__restrict__ mlmin, int32_t *__restrict__ father,
                             uint32_t *__restrict__ son, int *err) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const uint64_t k = key[t];
  const int l = ikey_lev(k);
  if (l <= mlmin[ikey_member(k)]) {
    father[t] = -1;
    return;
  }
  const uint32_t x = ikey_x(k), y = ikey_y(k), z = ikey_z(k);
  const int32_t v = hash_probe1(h, ikey_at(k, l - 1, x >> 1, y >> 1, z >> 1));
  if (v <= 0) {
    atomicOr(err, kErrGrading);
    father[t] = -1;
    return;
  }
  father[t] = v - 1;
  atomicOr(son + (v - 1), 1u << ((x & 1) | ((y & 1) << 1) | ((z & 1) << 2)));
}

// 27 level-(l-1) cells around the father cell of each oct above its
// member's levelmin (8-lane cooperative probes)
__global__ void k_grading(HashView h, const uint64_t *__restrict__ key, int64_t n,
                          const int *__restrict__ mlmin, int *err) {
  const int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 3;
  const int64_t t = q / 27;
  if (t >= n) return;
  const int e = int(q % 27);
  const uint64_t k = key[t];
  const int l = ikey_lev(k);
  if (l <= mlmin[ikey_member(k)]) return;  // the whole lane group leaves together
  const int64_t cells = int64_t(1) << (l - 1);
  const uint32_t x = wrapc(int64_t(ikey_x(k)) + (e % 3) - 1, cells);
  const uint32_t y = wrapc(int64_t(ikey_y(k)) + (e / 3 % 3) - 1, cells);
  const uint32_t z = wrapc(int64_t(ikey_z(k)) + (e / 9) - 1, cells);
  const int32_t v = hash_probe8(h, ikey_at(k, l - 1, x >> 1, y >> 1, z >> 1));
  if (v <= 0 && (threadIdx.x & 7) == 0) atomicOr(err, kErrGrading);
}

// ---------------------------------------------------------------------------
// 27-neighbour array; missing neighbours are claimed as ghost keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t neighbour_key(uint64_t k, int e) {
  const int l = ikey_lev(k);
  const int64_t side = int64_t(1) << (l - 1);
  return ikey_at(k, l, wrapc(int64_t(ikey_x(k)) + (e % 3) - 1, side),
                 wrapc(int64_t(ikey_y(k)) + (e / 3 % 3) - 1, side),
                 wrapc(int64_t(ikey_z(k)) + (e / 9) - 1, side));
}

__global__ void k_neighbours(HashView h, const uint64_t *__restrict__ key, int64_t n,
                             int32_t *__restrict__ nbr27, uint64_t *__restrict__ claim,
                             uint32_t *__restrict__ claim_count, int64_t claim_cap, int *err) {
  // one thread per (direction, oct), direction-major: coalesced table writes;
  // a query resolves in about one probe at this load factor, so each thread
  // probes alone (hash_probe8 would read 8 slots for it)
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 27 * n) return;
  const int e = int(q / n);
  const int64_t t = q - int64_t(e) * n;
  if (e == 13) {
    nbr27[q] = int32_t(t);
    return;
  }
  const uint64_t nk = neighbour_key(key[t], e);
  const int32_t v = hash_probe1(h, nk);
  if (v >= 1 && int64_t(v) <= n) {
    nbr27[q] = v - 1;
    return;
  }
  nbr27[q] = -1;
  bool ins = false;
  const uint64_t s = hash_insert(h, nk, &ins, err);
  if (ins && s != ~0ull) {
    h.val[s] = kPending;
    // one atomic per warp for its new claims (their order is sorted away)
    const unsigned grp = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(claim_count, uint32_t(__popc(grp)));
    base = __shfl_sync(grp, base, leader);
    const uint32_t slot = base + uint32_t(__popc(grp & ((1u << lane) - 1u)));
    if (int64_t(slot) < claim_cap)
      claim[slot] = nk;
    else
      atomicOr(err, kErrClaimOverflow);
  }
}

// compact sort key of a ghost key: (member, l, x, y, z), B bits per coordinate
__global__ void k_claim_to_comp(const uint64_t *__restrict__ claim, int64_t nc, int B,
                                uint64_t *__restrict__ comp, uint32_t *__restrict__ val) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nc) return;
  const uint64_t k = claim[t];
  comp[t] = (uint64_t(ikey_member(k)) << (4 + 3 * B)) | (uint64_t(ikey_lev(k)) << (3 * B)) |
            (uint64_t(ikey_x(k)) << (2 * B)) | (uint64_t(ikey_y(k)) << B) | uint64_t(ikey_z(k));
  val[t] = 0;
}

__global__ void k_cache_finalize(HashView h, const uint64_t *__restrict__ comp, int64_t nc, int B,
                                 int64_t N, uint64_t *__restrict__ ckey,
                                 uint32_t *__restrict__ seg_count, int *err) {
  const int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (s >= nc) return;
  const uint64_t c = comp[s];
  const uint64_t msk = (1ull << B) - 1;
  const int l = int((c >> (3 * B)) & 15);
  const int m = int(c >> (4 + 3 * B));
  const uint64_t k = ikey(m, l, uint32_t((c >> (2 * B)) & msk), uint32_t((c >> B) & msk), uint32_t(c & msk));
  ckey[s] = k;
  if (seg_count) warp_count(seg_count, 16 * m + l);
  uint64_t p = fnv1a64(k) & h.mask;
  for (uint64_t r = 0; r <= h.mask; ++r) {
    if (h.key[p] == k) {
      h.val[p] = int32_t(N + s + 1);
      return;
    }
    p = (p + 1) & h.mask;
  }
  atomicOr(err, kErrCacheMismatch);
}

__global__ void k_neighbours_fix(HashView h, const uint64_t *__restrict__ key, int64_t n,
                                 int32_t *__restrict__ nbr27, int *err) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 27 * n) return;
  if (nbr27[q] >= 0) return;
  const int e = int(q / n);
  const int64_t t = q - int64_t(e) * n;
  const int32_t v = hash_probe1(h, neighbour_key(key[t], e));
  if (v <= n || v == kPending) {
    atomicOr(err, kErrCacheMismatch);
    return;
  }
  nbr27[q] = v - 1;
}

// face-neighbour table of the extended oct range (real octs, then ghosts)
__global__ void k_faces_real(const int32_t *__restrict__ nbr27, int64_t n, int64_t next,
                             int32_t *__restrict__ fnb) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 6 * n) return;
  const int f = int(q / n);
  const int64_t t = q % n;
  fnb[int64_t(f) * next + t] = nbr27[int64_t(face_to_nbr27(f)) * n + t];
}

__global__ void k_faces_cache(HashView h, const uint64_t *__restrict__ ckey, int64_t nc, int64_t N,
                              int64_t next, int32_t *__restrict__ fnb) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= 6 * nc) return;
  const int f = int(q / nc);
  const int64_t s = q % nc;
  const int d = f >> 1, sg = (f & 1) ? 1 : -1;
  const int e = 13 + sg * (d == 0 ? 1 : (d == 1 ? 3 : 9));
  const int32_t v = hash_probe1(h, neighbour_key(ckey[s], e));
  fnb[int64_t(f) * next + N + s] = (v >= 1 && v != kPending) ? v - 1 : -1;
}

// cell of level L at cell coordinates (x,y,z) of member key km's mesh, or the
// coarser cell covering it when its oct is absent; -1 if none down to lmin.
__device__ int64_t cell_or_coarser(HashView h, uint64_t km, int L, int64_t x, int64_t y, int64_t z,
                                   int lmin, int64_t N, int *found_level) {
  while (L >= lmin) {
    const int64_t side = int64_t(1) << L;
    const uint32_t X = wrapc(x, side), Y = wrapc(y, side), Z = wrapc(z, side);
    const int32_t v = hash_probe1(h, ikey_at(km, L, X >> 1, Y >> 1, Z >> 1));
    if (v >= 1 && int64_t(v) <= N) {
      *found_level = L;
      return 8 * int64_t(v - 1) + ((X & 1) | ((Y & 1) << 1) | ((Z & 1) << 2));
    }
    x = X >> 1;
    y = Y >> 1;
    z = Z >> 1;
    --L;
  }
  return -1;
}

// prolongation sources of each ghost oct: its father cell C and C -/+ e_d
// for d = x, y, z (order C, -x, +x, -y, +y, -z, +z); C is also the coarse
// cell that receives the reflux of the ghost's faces (rslot[C] = ghost slot).
__global__ void k_cache_sources(HashView h, const uint64_t *__restrict__ ckey, int64_t nc, int64_t N,
                                const int *__restrict__ mlmin, int32_t *__restrict__ csrc,
                                int32_t *__restrict__ rslot, int *err) {
  const int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (s >= nc) return;
  const uint64_t k = ckey[s];
  const int l = ikey_lev(k);
  const int lmin = mlmin[ikey_member(k)];
  const int64_t x = ikey_x(k), y = ikey_y(k), z = ikey_z(k);
  for (int q = 0; q < 7; ++q) {
    const int d = (q - 1) >> 1;
    const int sg = (q & 1) ? -1 : 1;
    const int64_t dx = (q > 0 && d == 0) ? sg : 0, dy = (q > 0 && d == 1) ? sg : 0,
                  dz = (q > 0 && d == 2) ? sg : 0;
    int fl = -1;
    const int64_t c = cell_or_coarser(h, k, l - 1, x + dx, y + dy, z + dz, lmin, N, &fl);
    if (c < 0 || (q == 0 && fl != l - 1)) {
      atomicOr(err, kErrGrading);
      csrc[int64_t(q) * nc + s] = 0;
      continue;
    }
    csrc[int64_t(q) * nc + s] = int32_t(c);
    // distinct ghost octs have distinct fathers
    if (q == 0) rslot[c] = int32_t(s);
  }
}

// hash_get for a batch of internal keys (introspection), 8-lane groups
__global__ void k_lookup(HashView h, const uint64_t *__restrict__ keys, int64_t nq, int64_t N,
                         int64_t *__restrict__ out) {
  const int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 3;
  if (q >= nq) return;
  const int32_t v = hash_probe8(h, keys[q]);
  if ((threadIdx.x & 7) == 0) out[q] = (v >= 1 && int64_t(v) <= N) ? int64_t(v - 1) : -1;
}

// FNV-1a 64 of each value, by the function every hash insert and probe uses
__global__ void k_fnv(const uint64_t *__restrict__ in, int64_t n, uint64_t *__restrict__ out) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n) out[q] = fnv1a64(in[q]);
}

// Blocks of the fused kernels: runs of octs (mesh order) of one (member,
// level) whose coordinates lie in one aligned group of 2^sh octs per axis.
// head[o] = 1 where a block starts.
__global__ void k_block_heads(const uint64_t *__restrict__ key, int64_t n, unsigned sh,
                              uint32_t *__restrict__ head) {
  const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (o >= n) return;
  bool h = o == 0;
  if (!h) {
    const uint64_t k = key[o], q = key[o - 1];
    h = (k >> 45) != (q >> 45) || (ikey_x(k) >> sh) != (ikey_x(q) >> sh) ||
        (ikey_y(k) >> sh) != (ikey_y(q) >> sh) || (ikey_z(k) >> sh) != (ikey_z(q) >> sh);
  }
  head[o] = h ? 1u : 0u;
}

// first oct of every block (pos = exclusive prefix sum of head), and the end
// of the list after the last block
__global__ void k_block_starts(const uint32_t *__restrict__ head, const uint32_t *__restrict__ pos,
                               int64_t n, int32_t *__restrict__ start) {
  const int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (o >= n) return;
  if (head[o]) start[pos[o]] = int32_t(o);
  if (o == n - 1) start[pos[o] + head[o]] = int32_t(n);
}

// block of the octs ask[0..m)
__global__ void k_block_of(const uint32_t *__restrict__ head, const uint32_t *__restrict__ pos,
                           const int32_t *__restrict__ ask, int64_t m, int32_t *__restrict__ out) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m) return;
  const int32_t o = ask[t];
  out[t] = int32_t(pos[o] + head[o]) - 1;
}

}  // namespace amr
