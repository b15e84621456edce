// Sparse matrix -> MPO conversion (Alg. 4.1) in block form, on the GPU.
//
// Alg. 4.1 adds one rank-1 MPO per nonzero I1 x J1 block X of A: X on site 1 and unit
// matrices E_{i_k j_k} on sites 2..d (Section 4.1). The MPO rank is the number of nonzero
// blocks (Lemma 4.2), known before any value is written, so the conversion runs in two
// phases (Section 4.2: preallocation): count the blocks, then fill them.
//
// Input: COO (row, col, val) sorted by (row, col), no duplicates. Entries of block-row
// p = row / I1 form one contiguous segment. An entry is the "first occurrence" of its block
// (p, q), q = col / J1, when it is the first entry of its row with that q and no earlier row
// of the segment holds q (rows are sorted by col, so both tests are a neighbour compare and
// binary searches). Blocks are numbered in (p, q) order: block index t of a first occurrence
// = (#first occurrences before its segment) + (#distinct q' < q within the segment), the
// latter read off a prefix count F of first-occurrence flags with one binary search per row.
//
// Kernels:
//   k_first_scan  per entry: validate order/range, first-occurrence flag, tile-local exclusive
//                 scan of the flags (1024 entries per CTA) -> F_local, tile totals
//   k_tile_scan   one CTA: exclusive scan of the tile totals -> tile offsets, R
//   k_zero        zero X (vectorised)
//   k_fill_w      one warp per 32 consecutive entries: block index t of every entry (ranks
//                 among the first occurrences of its block-row, by shuffles inside the window),
//                 scatter the entry's value into block t, digits from each first occurrence.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tnr_internal.cuh"

namespace tnr {
namespace {

constexpr int kTile = 1024;

struct ConvDims {
  int64_t nrows, ncols, nnz;
  int64_t I1, J1;
  int32_t d;
  int32_t narrow;  // block-row indices fit 31 bits and block-column indices 30 (radix strides too)
  int32_t I[TNR_MAX_SITES];
  int32_t J[TNR_MAX_SITES];
  int32_t Is[TNR_MAX_SITES], Js[TNR_MAX_SITES];  // radix strides: prod of I_2..I_{k-1} (valid when narrow)
};

// Non-negative division that takes the 32-bit path whenever both operands fit (64-bit division
// is a long software sequence on the GPU; block and digit indices almost always fit).
__device__ __forceinline__ int64_t qdiv(int64_t a, int64_t b) {
  if ((((uint64_t)a) | ((uint64_t)b)) >> 32) return a / b;
  return (int64_t)((uint32_t)a / (uint32_t)b);
}

// Lower bound over entries [lo, hi) for the composite key (r, c).
__device__ __forceinline__ int64_t lower_bound_rc(const int64_t *__restrict__ row, const int64_t *__restrict__ col,
                                                  int64_t lo, int64_t hi, int64_t r, int64_t c) {
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    int64_t rm = __ldg(row + mid);
    bool less = rm < r || (rm == r && __ldg(col + mid) < c);
    if (less)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// First index in [0, e] whose row is >= rlo (entries sorted by row): gallop back from e.
__device__ __forceinline__ int64_t segment_start(const int64_t *__restrict__ row, int64_t e, int64_t rlo) {
  int64_t hi = e, step = 1, lo = e;
  while (true) {
    int64_t cand = e - step;
    if (cand < 0) {
      lo = 0;
      break;
    }
    if (__ldg(row + cand) < rlo) {
      lo = cand + 1;
      break;
    }
    hi = cand;
    step <<= 1;
  }
  // answer in [lo, hi]
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(row + mid) < rlo)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// First index in [e, nnz] whose row is >= rhi: gallop forward from e.
__device__ __forceinline__ int64_t segment_end(const int64_t *__restrict__ row, int64_t nnz, int64_t e, int64_t rhi) {
  int64_t lo = e, step = 1, hi = e;
  while (true) {
    int64_t cand = e + step;
    if (cand >= nnz) {
      hi = nnz;
      break;
    }
    if (__ldg(row + cand) >= rhi) {
      hi = cand;
      break;
    }
    lo = cand;
    step <<= 1;
  }
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(row + mid) < rhi)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Per entry: validation, first-occurrence flag of its block, tile-local exclusive scan of the flags.
// An entry of row r > p I1 is the first of block (p, q) when no earlier row of block-row p holds a
// column in [q J1, (q+1) J1). The tile's rows and columns are staged in shared memory, so that
// test is a few binary searches in shared memory whenever the block-row's segment starts inside the
// tile (a segment crossing the tile's start falls back to searches in global memory). seg (may be
// null): seg[pp] = first entry of block-row pp, for pp < seg_len (seg[seg_len - 1] = nnz).
constexpr int kHalo = 128;  // entries before the tile staged with it (block-rows crossing the tile start)

__global__ void __launch_bounds__(kTile, 2) k_first_scan(const int64_t *__restrict__ row, const int64_t *__restrict__ col,
                                                      ConvDims D, int32_t *__restrict__ F_local,
                                                      int32_t *__restrict__ tile_total, int32_t *__restrict__ seg,
                                                      int64_t seg_len, int *status) {
  __shared__ int32_t warp_sums[kTile / 32];
  __shared__ int64_t s_row[kHalo + kTile], s_col[kHalo + kTile];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  const int64_t e = base + threadIdx.x;
  const int64_t hbase = base > kHalo ? base - kHalo : 0;  // first staged entry
  const int hoff = (int)(base - hbase);                    // local index of entry `base`
  for (int i = threadIdx.x; i < hoff + kTile; i += kTile) {
    const int64_t x = hbase + i;
    if (x < D.nnz) {
      s_row[i] = __ldg(row + x);
      s_col[i] = __ldg(col + x);
    }
  }
  __syncthreads();
  const int me = hoff + (int)threadIdx.x;  // local index of entry e
  int flag = 0;
  if (e < D.nnz) {
    const int64_t r = s_row[me], c = s_col[me];
    const int64_t rp = e == 0 ? -1 : s_row[me - 1];
    const int64_t cp = e == 0 ? -1 : s_col[me - 1];
    bool ok = true;
    if (r < 0 || r >= D.nrows || c < 0 || c >= D.ncols) {
      set_status(status, TNR_ERANGE);
      ok = false;
    }
    if (e > 0) {
      if (rp > r || (rp == r && cp > c)) {
        set_status(status, TNR_ENOTSORTED);
        ok = false;
      } else if (rp == r && cp == c) {
        set_status(status, TNR_EDUP);
        ok = false;
      }
    }
    if (ok) {
      const int64_t p = qdiv(r, D.I1), q = qdiv(c, D.J1);
      const int64_t r0 = p * D.I1, clo = q * D.J1, chi = (q + 1) * D.J1;
      bool first = !(e > 0 && rp == r && qdiv(cp, D.J1) == q);
      if (first && r > r0) {
        // does block-row p start inside the staged range?
        const bool inside = hbase == 0 || s_row[0] < r0;
        // short block-row prefix: walk back over the earlier rows' entries (the same row's
        // entries with the same block-column are adjacent, handled above)
        int i = me - 1, steps = 0;
        bool walked = false;
        if (inside) {
          while (i >= 0 && s_row[i] == r) --i;
          for (; i >= 0 && steps < 96; --i, ++steps) {
            if (s_row[i] < r0) break;
            if (s_col[i] >= clo && s_col[i] < chi) {
              first = false;
              break;
            }
          }
          walked = !first || i < 0 || s_row[i] < r0;
        }
        if (walked) {
          // decided by the walk
        } else if (inside) {
          int lo = 0, hi = me;  // first local index with row >= r0
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_row[mid] < r0)
              lo = mid + 1;
            else
              hi = mid;
          }
          for (int64_t rr = r0; rr < r && first; ++rr) {
            int a = lo, b = me;  // first index in [lo, me) with (row, col) >= (rr, clo)
            while (a < b) {
              const int mid = (a + b) >> 1;
              if (s_row[mid] < rr || (s_row[mid] == rr && s_col[mid] < clo))
                a = mid + 1;
              else
                b = mid;
            }
            if (a < me && s_row[a] == rr && s_col[a] < chi) first = false;
            lo = a;
          }
        } else {
          const int64_t s0 = segment_start(row, e, r0);
          for (int64_t rr = r0; rr < r && first; ++rr) {
            const int64_t x = lower_bound_rc(row, col, s0, e, rr, clo);
            if (x < e && __ldg(row + x) == rr && __ldg(col + x) < chi) first = false;
          }
        }
      }
      flag = first ? 1 : 0;
      if (seg) {  // starts of the block-rows between the previous entry's and this one's
        const int64_t pprev = e == 0 ? -1 : qdiv(rp, D.I1);
        for (int64_t pp = pprev + 1; pp <= p && pp < seg_len; ++pp) seg[pp] = (int32_t)e;
        if (e == D.nnz - 1)
          for (int64_t pp = p + 1; pp < seg_len; ++pp) seg[pp] = (int32_t)D.nnz;
      }
    }
  }
  // CTA-wide exclusive scan of flag.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = flag;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = warp_sums[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    warp_sums[lane] = wi - w;  // exclusive prefix of warp totals
    if (lane == 31) tile_total[blockIdx.x] = wi;
  }
  __syncthreads();
  if (e < D.nnz) F_local[e] = warp_sums[warp] + incl - flag;
}

// Exclusive scan of the tile totals in place; writes the grand total to tile_off[ntiles].
__global__ void __launch_bounds__(1024) k_tile_scan(int32_t *__restrict__ tile_off, int64_t ntiles) {
  __shared__ int32_t warp_sums[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < ntiles; base += 1024) {
    const int64_t i = base + threadIdx.x;
    int v = i < ntiles ? tile_off[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int w = warp_sums[lane], wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += u;
      }
      warp_sums[lane] = wi - w;
    }
    __syncthreads();
    const int c0 = carry;
    if (i < ntiles) tile_off[i] = c0 + warp_sums[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c0 + warp_sums[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_off[ntiles] = carry;
}

__device__ __forceinline__ int64_t F_at(const int32_t *__restrict__ F_local, const int32_t *__restrict__ tile_off,
                                        int64_t x, int64_t nnz) {
  if (x >= nnz) return tile_off[cdiv(nnz, kTile)];
  return (int64_t)__ldg(tile_off + x / kTile) + __ldg(F_local + x);
}

// Digits of block t: i_k, j_k of the block-row p and block-column q (mixed radix, site 2 fastest).
__device__ __forceinline__ void write_digits(const ConvDims &D, int64_t p, int64_t q, int64_t t, uint8_t *digits) {
  if (D.d <= 1) return;
  uint8_t *dg = digits + t * 2 * (int64_t)(D.d - 1);
  int64_t pp = p, qq = q;
  for (int k = 1; k < D.d; ++k) {
    const int64_t pq = qdiv(pp, D.I[k]), qq2 = qdiv(qq, D.J[k]);
    dg[2 * (k - 1)] = (uint8_t)(pp - pq * D.I[k]);
    dg[2 * (k - 1) + 1] = (uint8_t)(qq - qq2 * D.J[k]);
    pp = pq;
    qq = qq2;
  }
}

// Segments handled whole by k_fill_rows: at most two entries per lane, blocks within the warp's buffer.
constexpr int kRowsMaxL = 64;
constexpr int kRowsBuf = 512;  // doubles of shared buffer per warp (4 KB)
constexpr int kRowsDig = 1024;  // bytes of digit staging per warp
__device__ __forceinline__ bool fill_rows_small(int64_t L, int64_t nb, int64_t bs) {
  return L <= kRowsMaxL && nb * bs <= kRowsBuf;
}

// Warp-window fill. Warp w handles the 32 consecutive nonzeros [32w, 32w + 32). Lanes whose
// entries share a block-row p form a run (entries are sorted, so runs are contiguous lanes and
// found with a ballot). The block index of an entry is t = F(s0) + rank, rank = number of first
// occurrences in its block-row segment [s0, s1) with a smaller block-column; inside the window
// it is counted with shuffles, outside it (only for the runs that cross a window edge) with a
// linear scan of the segment's remaining entries. X is zeroed beforehand (k_zero), so every
// nonzero writes its own value and the first occurrence of each block also writes its digits.
__global__ void __launch_bounds__(256) k_zero(double *__restrict__ X, int64_t n) {
  if (reinterpret_cast<uintptr_t>(X) & 15) {  // not 16-byte aligned: scalar stores
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      X[i] = 0.0;
    return;
  }
  const int64_t n2 = n >> 1;
  double2 *X2 = reinterpret_cast<double2 *>(X);
  const double2 z = make_double2(0.0, 0.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
    X2[i] = z;
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) X[n - 1] = 0.0;
}

__global__ void __launch_bounds__(256) k_fill_w(const int64_t *__restrict__ row, const int64_t *__restrict__ col,
                                                const double *__restrict__ val, ConvDims D,
                                                const int32_t *__restrict__ F_local,
                                                const int32_t *__restrict__ tile_off, double *__restrict__ X,
                                                uint8_t *__restrict__ digits, int64_t R,
                                                const int32_t *__restrict__ seg, const int *__restrict__ big,
                                                int *status) {
  const int lane = threadIdx.x & 31;
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;  // window start
  if (e0 >= D.nnz) return;
  if (big && *big == 0) return;  // k_fill_rows wrote every block-row
  const int64_t e = e0 + lane;
  const bool valid = e < D.nnz;
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);
  const int nval = __popc(vmask);
  int64_t r = -1, c = 0, p = -1, q = 0;
  int first = 0;
  double v = 0.0;
  if (valid) {
    r = __ldg(row + e);
    c = __ldg(col + e);
    v = __ldg(val + e);
    p = qdiv(r, D.I1);
    q = qdiv(c, D.J1);
    first = F_at(F_local, tile_off, e + 1, D.nnz) != F_at(F_local, tile_off, e, D.nnz);
  }
  // runs of equal block-row across lanes
  const int64_t pprev = __shfl_up_sync(0xffffffffu, p, 1);
  const bool bound = valid && (lane == 0 || pprev != p);
  const unsigned bmask = __ballot_sync(0xffffffffu, bound);
  const int rs = 31 - __clz(bmask & (0xffffffffu >> (31 - lane)));     // run start lane
  const unsigned after = bmask & ~(0xffffffffu >> (31 - lane));         // boundaries after me
  const int re = after ? (__ffs(after) - 2) : (nval - 1);               // run end lane
  // segment bounds: gallop only where the run touches the window edge
  int64_t s0 = e0 + rs, s1 = e0 + re + 1;
  const int64_t r0 = p * D.I1;
  if (valid && rs == 0 && e0 > 0 && qdiv(__ldg(row + e0 - 1), D.I1) == p) s0 = segment_start(row, e0, r0);
  if (valid && re == nval - 1 && e0 + nval < D.nnz && qdiv(__ldg(row + e0 + nval), D.I1) == p)
    s1 = segment_end(row, D.nnz, e0 + nval - 1, r0 + D.I1);
  // rank inside the window (lanes rs..re of my run)
  int64_t rank = 0;
  for (int j = 0; j < 32; ++j) {
    const int64_t qj = __shfl_sync(0xffffffffu, q, j);
    const int fj = __shfl_sync(0xffffffffu, first, j);
    if (valid && j >= rs && j <= re && fj && qj < q) ++rank;
  }
  // rank outside the window, for runs crossing an edge
  if (valid) {
    for (int64_t x = s0; x < e0 + rs; ++x)
      if (qdiv(__ldg(col + x), D.J1) < q && F_at(F_local, tile_off, x + 1, D.nnz) != F_at(F_local, tile_off, x, D.nnz))
        ++rank;
    for (int64_t x = e0 + re + 1; x < s1; ++x)
      if (qdiv(__ldg(col + x), D.J1) < q && F_at(F_local, tile_off, x + 1, D.nnz) != F_at(F_local, tile_off, x, D.nnz))
        ++rank;
    const int64_t t = F_at(F_local, tile_off, s0, D.nnz) + rank;
    if (t < 0 || t >= R) {
      set_status(status, TNR_ERANGE);
      return;
    }
    if (seg && fill_rows_small(s1 - s0, F_at(F_local, tile_off, s1, D.nnz) - F_at(F_local, tile_off, s0, D.nnz),
                               D.I1 * D.J1))
      return;  // written by k_fill_rows
    X[t * D.I1 * D.J1 + (r - r0) + D.I1 * (c - q * D.J1)] = v;
    if (first) write_digits(D, p, q, t, digits);
  }
}

// Block-row fill, one warp per block-row p with segment [seg[p], seg[p+1]). A short segment (at
// most kRowsMaxL entries, its blocks at most kRowsBuf values) is assembled in the warp's shared
// buffer (zeros, then each entry's value at its block's rank among the block-row's distinct
// block-columns) and written out whole, block after block, with its digits; no block of X is
// touched twice and every write covers whole sectors. A longer segment only has its blocks zeroed
// here (coalesced) and raises *big; k_fill_w then scatters its values and digits.
__global__ void __launch_bounds__(256) k_fill_rows(const int64_t *__restrict__ row, const int64_t *__restrict__ col,
                                                   const double *__restrict__ val, ConvDims D,
                                                   const int32_t *__restrict__ F_local,
                                                   const int32_t *__restrict__ tile_off,
                                                   const int32_t *__restrict__ seg, int64_t nbr,
                                                   double *__restrict__ X, uint8_t *__restrict__ digits, int64_t R,
                                                   int *big, int *status) {
  __shared__ double s_buf[8][kRowsBuf];
  __shared__ uint8_t s_dig[8][kRowsDig];
  __shared__ uint8_t s_pdig[8][TNR_MAX_SITES];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  double *buf = s_buf[wl];
  const int64_t bs = D.I1 * D.J1;
  const int64_t nd = 2 * (int64_t)(D.d - 1);  // digit bytes per block
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < nbr;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t s0 = seg[p], s1 = seg[p + 1], L = s1 - s0;
    if (L <= 0) continue;
    const int64_t t0 = F_at(F_local, tile_off, s0, D.nnz);
    const int64_t nb = F_at(F_local, tile_off, s1, D.nnz) - t0;
    if (t0 < 0 || nb < 1 || t0 + nb > R) {
      if (lane == 0) set_status(status, TNR_ERANGE);
      continue;
    }
    if (!fill_rows_small(L, nb, bs)) {  // long segment: zero its blocks, k_fill_w scatters
      for (int64_t i = lane; i < nb * bs; i += 32) X[t0 * bs + i] = 0.0;
      if (lane == 0) atomicOr(big, 1);
      continue;
    }
    const int64_t r0 = p * D.I1;
    int64_t rr[2], qq[2];
    double vv[2];
    int ff[2];
    bool have[2];
    for (int h = 0; h < 2; ++h) {
      const int64_t e = s0 + lane + 32 * h;
      have[h] = e < s1;
      rr[h] = have[h] ? __ldg(row + e) : 0;
      const int64_t c = have[h] ? __ldg(col + e) : 0;
      qq[h] = have[h] ? qdiv(c, D.J1) : 0;
      vv[h] = have[h] ? __ldg(val + e) : 0.0;
      ff[h] = have[h] ? (F_at(F_local, tile_off, e + 1, D.nnz) != F_at(F_local, tile_off, e, D.nnz)) : 0;
      rr[h] = rr[h] - r0 + D.I1 * (c - qq[h] * D.J1);  // offset inside the block
    }
    // rank of each entry's block: distinct block-columns of the segment below its own
    int64_t rank[2] = {0, 0};
    if (D.narrow) {  // block columns and first flags packed in one 32-bit word (q < 2^31)
      const int32_t w0 = ((int32_t)qq[0] << 1) | ff[0], w1 = ((int32_t)qq[1] << 1) | ff[1];
      const int32_t m0 = (int32_t)qq[0] << 1, m1 = (int32_t)qq[1] << 1;
      int r0c = 0, r1c = 0;
      for (int j = 0; j < (int)L; ++j) {
        const int32_t wj = __shfl_sync(0xffffffffu, (j >> 5) ? w1 : w0, j & 31);
        // first occurrence (low bit) with a smaller block column
        r0c += ((wj & 1) && wj < m0) ? 1 : 0;
        r1c += ((wj & 1) && wj < m1) ? 1 : 0;
      }
      rank[0] = r0c;
      rank[1] = r1c;
    } else {
      for (int j = 0; j < (int)L; ++j) {
        const int hj = j >> 5, lj = j & 31;
        const int64_t qj = __shfl_sync(0xffffffffu, hj ? qq[1] : qq[0], lj);
        const int fj = __shfl_sync(0xffffffffu, hj ? ff[1] : ff[0], lj);
        for (int h = 0; h < 2; ++h)
          if (fj && qj < qq[h]) ++rank[h];
      }
    }
    for (int64_t i = lane; i < nb * bs; i += 32) buf[i] = 0.0;
    __syncwarp();
    for (int h = 0; h < 2; ++h)
      if (have[h]) buf[rank[h] * bs + rr[h]] = vv[h];
    __syncwarp();
    for (int64_t i = lane; i < nb * bs; i += 32) X[t0 * bs + i] = buf[i];
    if (nd > 0 && nb * nd <= kRowsDig) {  // the block-row's digit rows are contiguous: stage, then
      uint8_t *dg = s_dig[wl];             // one run of consecutive byte stores
      if (D.narrow) {
        // digit k of p (shared by every block of the block-row) and of each block's q from the
        // radix strides: independent 32-bit divisions instead of a dependent chain
        const uint32_t p32 = (uint32_t)p;
        for (int k = 1 + lane; k < D.d; k += 32) s_pdig[wl][k] = (uint8_t)((p32 / (uint32_t)D.Is[k]) % (uint32_t)D.I[k]);
        __syncwarp();
        for (int h = 0; h < 2; ++h) {
          if (!(have[h] && ff[h])) continue;
          const uint32_t q32 = (uint32_t)qq[h];
          uint8_t *row_d = dg + rank[h] * nd;
          for (int k = 1; k < D.d; ++k) {
            row_d[2 * (k - 1)] = s_pdig[wl][k];
            row_d[2 * (k - 1) + 1] = (uint8_t)((q32 / (uint32_t)D.Js[k]) % (uint32_t)D.J[k]);
          }
        }
      } else {
        for (int h = 0; h < 2; ++h)
          if (have[h] && ff[h]) write_digits(D, p, qq[h], rank[h], dg);
      }
      __syncwarp();
      for (int64_t i = lane; i < nb * nd; i += 32) digits[t0 * nd + i] = dg[i];
    } else {
      for (int h = 0; h < 2; ++h)
        if (have[h] && ff[h]) write_digits(D, p, qq[h], t0 + rank[h], digits);
    }
    __syncwarp();
  }
}

int make_dims(int64_t nrows, int64_t ncols, int64_t nnz, int32_t d, const int64_t *I, const int64_t *J, ConvDims *D) {
  if (d < 1 || d > TNR_MAX_SITES || !I || !J || nrows < 1 || ncols < 1 || nnz < 0) return TNR_EINVAL;
  if (nnz >= (int64_t(1) << 31)) return TNR_ERANGE;
  __int128 pi = 1, pj = 1;
  for (int k = 0; k < d; ++k) {
    if (I[k] < 1 || J[k] < 1) return TNR_EINVAL;
    if (k > 0 && (I[k] > 256 || J[k] > 256)) return TNR_EINVAL;
    pi *= I[k];
    pj *= J[k];
    if (pi > ((__int128)1 << 62) || pj > ((__int128)1 << 62)) return TNR_EINVAL;
    D->I[k] = (int32_t)(k > 0 ? I[k] : 0);
    D->J[k] = (int32_t)(k > 0 ? J[k] : 0);
  }
  if (pi != nrows || pj != ncols) return TNR_EINVAL;
  if (I[0] * J[0] > 4096) return TNR_EINVAL;
  {
    const int64_t lim = (int64_t(1) << 31) - 1;
    // block rows below 2^31, block columns below 2^30 (the fill packs 2 q + flag in 32 bits)
    D->narrow = (nrows / I[0] <= lim && ncols / J[0] <= (lim >> 1)) ? 1 : 0;
    int64_t si = 1, sj = 1;
    for (int k = 1; k < d; ++k) {
      D->Is[k] = (int32_t)(si <= lim ? si : 0);
      D->Js[k] = (int32_t)(sj <= lim ? sj : 0);
      si *= I[k];
      sj *= J[k];
    }
  }
  D->nrows = nrows;
  D->ncols = ncols;
  D->nnz = nnz;
  D->I1 = I[0];
  D->J1 = J[0];
  D->d = d;
  return TNR_OK;
}

size_t ws_bytes_for(int64_t nnz) {
  const int64_t ntiles = cdiv(nnz, kTile);
  return ((size_t(nnz) * 4 + 255) & ~size_t(255)) + ((size_t(ntiles + 1) * 4 + 255) & ~size_t(255));
}

// Block-row segment starts (one int32 per block-row, plus the end) are kept when the number of
// block-rows is modest next to nnz; then the fill writes whole blocks (k_fill_rows).
int64_t seg_len_for(int64_t nrows, int64_t I1, int64_t nnz) {
  const int64_t nbr = nrows / I1;
  return nbr <= 4 * nnz + (int64_t(1) << 20) ? nbr + 1 : 0;
}

// Workspace of the two-phase conversion: F_local | tile offsets | segment starts | the long-segment flag.
struct ConvWs {
  int32_t *F_local, *tile_off, *seg;
  int *big;
  int64_t seg_len;
};
size_t conv_ws_bytes(int64_t nrows, int64_t I1, int64_t nnz) {
  const int64_t sl = seg_len_for(nrows, I1, nnz);
  return ws_bytes_for(nnz) + ((size_t(sl) * 4 + 255) & ~size_t(255)) + 256;
}
ConvWs conv_ws(void *ws, int64_t nrows, int64_t I1, int64_t nnz) {
  ConvWs w;
  char *b = static_cast<char *>(ws);
  w.F_local = reinterpret_cast<int32_t *>(b);
  w.tile_off = reinterpret_cast<int32_t *>(b + ((size_t(nnz) * 4 + 255) & ~size_t(255)));
  w.seg_len = seg_len_for(nrows, I1, nnz);
  w.seg = w.seg_len ? reinterpret_cast<int32_t *>(b + ws_bytes_for(nnz)) : nullptr;
  w.big = reinterpret_cast<int *>(b + ws_bytes_for(nnz) + ((size_t(w.seg_len) * 4 + 255) & ~size_t(255)));
  return w;
}

}  // namespace
}  // namespace tnr

using namespace tnr;

extern "C" int tnr_sparse_workspace(int64_t nrows, int64_t ncols, int64_t nnz, int32_t d, const int64_t *I,
                                    const int64_t *J, size_t *bytes) {
  ConvDims D;
  TNR_TRY(make_dims(nrows, ncols, nnz, d, I, J, &D));
  if (!bytes) return TNR_EINVAL;
  *bytes = conv_ws_bytes(nrows, I[0], nnz);
  return TNR_OK;
}

extern "C" int tnr_sparse_count(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row, const int64_t *col,
                                int32_t d, const int64_t *I, const int64_t *J, int64_t *R_out, void *ws,
                                size_t ws_bytes, void *stream) {
  ConvDims D;
  TNR_TRY(make_dims(nrows, ncols, nnz, d, I, J, &D));
  if (!R_out) return TNR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (nnz == 0) {
    *R_out = 0;
    return TNR_OK;
  }
  if (!row || !col || !ws) return TNR_EINVAL;
  if (ws_bytes < conv_ws_bytes(nrows, I[0], nnz)) return TNR_ENOMEM;
  const int64_t ntiles = cdiv(nnz, kTile);
  const ConvWs W = conv_ws(ws, nrows, I[0], nnz);
  int32_t *F_local = W.F_local, *tile_off = W.tile_off;
  TNR_TRY(reset_status(s));
  {
    LaunchScope ls(K_CONV_FLAGS, s);
    k_first_scan<<<(unsigned)ntiles, kTile, 0, s>>>(row, col, D, F_local, tile_off, W.seg, W.seg_len, status_ptr());
  }
  TNR_CK(cudaGetLastError());
  {
    LaunchScope ls(K_CONV_SCAN, s);
    k_tile_scan<<<1, 1024, 0, s>>>(tile_off, ntiles);
  }
  TNR_CK(cudaGetLastError());
  int32_t total = 0;
  const ReadBack rb[1] = {{&total, tile_off + ntiles, sizeof(int32_t)}};
  int st = read_back(s, rb, 1);  // synchronises once
  if (st != TNR_OK) return st;
  *R_out = total;
  return TNR_OK;
}

extern "C" int tnr_sparse_fill(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row, const int64_t *col,
                               const double *val, int32_t d, const int64_t *I, const int64_t *J, int64_t R,
                               double *X, uint8_t *digits, void *ws, size_t ws_bytes, void *stream) {
  ConvDims D;
  TNR_TRY(make_dims(nrows, ncols, nnz, d, I, J, &D));
  if (nnz == 0 || R == 0) return TNR_OK;
  if (!row || !col || !val || !X || !ws || (d > 1 && !digits) || R < 0) return TNR_EINVAL;
  if (ws_bytes < conv_ws_bytes(nrows, I[0], nnz)) return TNR_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const ConvWs W = conv_ws(ws, nrows, I[0], nnz);
  const int32_t *F_local = W.F_local, *tile_off = W.tile_off;
  // algorithmic bytes of the conversion: 24 B per nonzero read, values and digits written
  stats_work(K_CONV_FILL, 24.0 * (double)nnz + (double)R * (8.0 * (double)(I[0] * J[0]) + 2.0 * (d - 1)));
  if (W.seg) {  // whole blocks per block-row; the scatter kernel only for long segments (if any)
    const int64_t nbr = W.seg_len - 1;
    TNR_CK(cudaMemsetAsync(W.big, 0, sizeof(int), s));
    {
      LaunchScope ls(K_CONV_FILL, s);
      k_fill_rows<<<(unsigned)std::min<int64_t>(cdiv(nbr, 8), 152 * 64), 256, 0, s>>>(
          row, col, val, D, F_local, tile_off, W.seg, nbr, X, digits, R, W.big, status_ptr());
    }
    {
      LaunchScope ls(K_CONV_FILL, s);
      k_fill_w<<<(unsigned)cdiv(nnz, 256), 256, 0, s>>>(row, col, val, D, F_local, tile_off, X, digits, R, W.seg,
                                                         W.big, status_ptr());
    }
    TNR_CK(cudaGetLastError());
    return TNR_OK;
  }
  {
    LaunchScope ls(K_CONV_FILL, s);
    const int64_t nx = R * I[0] * J[0];
    k_zero<<<(unsigned)std::min<int64_t>(cdiv(nx / 2 + 1, 256), 152 * 16), 256, 0, s>>>(X, nx);
  }
  {
    LaunchScope ls(K_CONV_FILL, s);
    k_fill_w<<<(unsigned)cdiv(nnz, 256), 256, 0, s>>>(row, col, val, D, F_local, tile_off, X, digits, R, nullptr,
                                                       nullptr, status_ptr());
  }
  TNR_CK(cudaGetLastError());
  return TNR_OK;
}

// ---------------------------------------------------------------------------------------------
// Dense cores of the Alg. 4.1 MPO (Section 4.1: the sum of the rank-1 MPOs E_{i_d j_d} (x) ... (x)
// E_{i_2 j_2} (x) X_t has rank R at every bond, Lemma 4.2). Site 1 holds the blocks themselves
// (core (0, i1, j1, t) = X_t(i1, j1): the same memory as X); site k (2..d-1) is a bond-diagonal
// selection, core (t, i, j, t) = [i = i_{t,k}][j = j_{t,k}]; site d is (t, i, j, 0) = [...]. The
// cores are zeroed first, then one thread per (block, site) writes its single 1.0. For d = 1 the
// one core is the sum of the blocks. Copy and integer work only: bit-exact.
// ---------------------------------------------------------------------------------------------
struct CoreSites {
  double *core[TNR_MAX_SITES];
  int32_t I[TNR_MAX_SITES], J[TNR_MAX_SITES];
};

__global__ void __launch_bounds__(256) k_block_units(const uint8_t *__restrict__ digits, int64_t R, int32_t d,
                                                     const __grid_constant__ CoreSites S, int *status) {
  const int64_t total = R * (d - 1);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx % R;
    const int k = 1 + (int)(idx / R);
    const int i = digits[t * 2 * (d - 1) + 2 * (k - 1)], j = digits[t * 2 * (d - 1) + 2 * (k - 1) + 1];
    const int I = S.I[k], J = S.J[k];
    if (i >= I || j >= J) {
      set_status(status, TNR_ERANGE);
      continue;
    }
    const int64_t r2 = k == d - 1 ? 0 : t;  // the last site closes the bond
    S.core[k][t + R * (i + (int64_t)I * (j + (int64_t)J * r2))] = 1.0;
  }
}

__global__ void __launch_bounds__(256) k_block_sum(const double *__restrict__ X, int64_t R, int64_t bs,
                                                   double *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < bs; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t t = 0; t < R; ++t) acc += X[t * bs + e];  // blocks in order
    out[e] = acc;
  }
}

// ---------------------------------------------------------------------------------------------
// Conversion without any device allocation (no counterpart in the paper).
//
// The scratch that tnr_sparse_count/fill take from the caller's workspace (one int32 prefix
// count per nonzero plus one int32 per 1024-entry tile) lives here in a file-scope device array
// instead, sized for TNR_NOALLOC_MAX_NNZ nonzeros (32 MiB + 32 KiB). Every GPU that loads the
// library holds this array until the process exits. Host code must not hand the array's name
// to a kernel (in host code it is only a stand-in symbol); its device address is looked up
// once per device with cudaGetSymbolAddress while that device is current, on the first call
// made on that device. Nothing in the array has to start at zero: each call writes every
// entry it later reads. All calls share the array, so calls whose kernels overlap on the GPU
// (different streams, or different host threads on the same device) race.
// ---------------------------------------------------------------------------------------------
namespace tnr {
namespace {

constexpr int64_t kNoAllocTiles = (TNR_NOALLOC_MAX_NNZ + kTile - 1) / kTile;
static __device__ __align__(256) int32_t g_noalloc_scratch[TNR_NOALLOC_MAX_NNZ + kNoAllocTiles + 64];

std::mutex g_noalloc_mu;
int32_t *g_noalloc_ptr[kMaxDevices] = {nullptr};  // per device ordinal

int noalloc_scratch(int32_t **out) {
  int dev = 0;
  TNR_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return TNR_ERANGE;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    TNR_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return TNR_OK;
}

}  // namespace
}  // namespace tnr

extern "C" int tnr_sparse_to_mpo_noalloc(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row,
                                         const int64_t *col, const double *val, int32_t d, const int64_t *I,
                                         const int64_t *J, double *X, uint8_t *digits, int64_t max_blocks,
                                         int64_t *R_out, void *stream) {
  ConvDims D;
  TNR_TRY(make_dims(nrows, ncols, nnz, d, I, J, &D));
  if (!R_out || max_blocks < 0) return TNR_EINVAL;
  if (nnz > TNR_NOALLOC_MAX_NNZ) return TNR_ERANGE;
  if (nnz == 0) {
    *R_out = 0;
    return TNR_OK;
  }
  if (!row || !col || !val || !X || (d > 1 && !digits)) return TNR_EINVAL;
  int32_t *scratch = nullptr;
  TNR_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ntiles = cdiv(nnz, kTile);
  int32_t *F_local = scratch;
  int32_t *tile_off = scratch + TNR_NOALLOC_MAX_NNZ;
  TNR_TRY(reset_status(s));
  {
    LaunchScope ls(K_CONV_FLAGS, s);
    k_first_scan<<<(unsigned)ntiles, kTile, 0, s>>>(row, col, D, F_local, tile_off, nullptr, 0, status_ptr());
  }
  TNR_CK(cudaGetLastError());
  {
    LaunchScope ls(K_CONV_SCAN, s);
    k_tile_scan<<<1, 1024, 0, s>>>(tile_off, ntiles);
  }
  TNR_CK(cudaGetLastError());
  int32_t total = 0;
  const ReadBack rb[1] = {{&total, tile_off + ntiles, sizeof(int32_t)}};
  int st = read_back_unstaged(s, rb, 1);  // synchronises once; no pinned staging buffer
  if (st != TNR_OK) return st;
  *R_out = total;
  if (total > max_blocks) return TNR_ENOMEM;  // X and digits untouched
  {
    LaunchScope ls(K_CONV_FILL, s);
    const int64_t nx = total * I[0] * J[0];
    k_zero<<<(unsigned)std::min<int64_t>(cdiv(nx / 2 + 1, 256), 152 * 16), 256, 0, s>>>(X, nx);
  }
  {
    LaunchScope ls(K_CONV_FILL, s);
    k_fill_w<<<(unsigned)cdiv(nnz, 256), 256, 0, s>>>(row, col, val, D, F_local, tile_off, X, digits, total,
                                                       nullptr, nullptr, status_ptr());
  }
  TNR_CK(cudaGetLastError());
  return TNR_OK;
}

extern "C" int tnr_sparse_cores(int64_t R, const double *X, const uint8_t *digits, int32_t d, const int64_t *I,
                                const int64_t *J, tnr_mpo *A, void *stream) {
  if (!A || d < 1 || d > TNR_MAX_SITES || !I || !J || R < 1 || !X || (d > 1 && !digits)) return TNR_EINVAL;
  for (int k = 0; k < d; ++k) {
    if (I[k] < 1 || J[k] < 1 || (k > 0 && (I[k] > 256 || J[k] > 256))) return TNR_EINVAL;
    if (!A->core[k]) return TNR_EINVAL;
  }
  const int64_t bs = I[0] * J[0];
  if (bs > 4096 || R > (int64_t(1) << 31)) return TNR_ERANGE;
  A->d = d;
  A->dtype = TNR_F64;
  A->R[0] = 1;
  A->R[d] = 1;
  for (int k = 1; k < d; ++k) A->R[k] = R;
  for (int k = 0; k < d; ++k) {
    A->I[k] = I[k];
    A->J[k] = J[k];
    const double need = (double)A->R[k] * (double)I[k] * (double)J[k] * (double)A->R[k + 1];
    if (need > (double)A->cap[k]) return TNR_ENOMEM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  LaunchScope ls(K_CONV_FILL, s);
  if (d == 1) {
    k_block_sum<<<(unsigned)std::min<int64_t>(cdiv(bs, 256), 4096), 256, 0, s>>>(X, R, bs, A->core[0]);
    return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
  }
  TNR_CK(cudaMemcpyAsync(A->core[0], X, sizeof(double) * R * bs, cudaMemcpyDeviceToDevice, s));
  CoreSites S;
  memset(&S, 0, sizeof(S));
  for (int k = 1; k < d; ++k) {
    const int64_t n = A->R[k] * I[k] * J[k] * A->R[k + 1];
    TNR_CK(cudaMemsetAsync(A->core[k], 0, sizeof(double) * n, s));
    S.core[k] = A->core[k];
    S.I[k] = (int32_t)I[k];
    S.J[k] = (int32_t)J[k];
  }
  const int64_t total = R * (d - 1);
  k_block_units<<<(unsigned)std::min<int64_t>(cdiv(total, 256), 152 * 16), 256, 0, s>>>(digits, R, d, S,
                                                                                      status_ptr());
  return check_cuda_at(cudaGetLastError(), __FILE__, __LINE__);
}
