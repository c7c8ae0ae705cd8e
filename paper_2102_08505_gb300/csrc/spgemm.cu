// spgemm.cu -- thresholded ELLPACK matrix-matrix multiply and add.
//
// C = drop_tau(alpha * A*B + beta * Add): the "ELLPACK X2" operation of Section
// "Performance Evaluation using System Matrices" with the "SP2 Loop Misc" update fused
// into its epilogue (Section "Performance Evaluation using an ExaSP2 Application").
//
// Design (GB300).  Row-wise Gustavson: output row i accumulates alpha * a_ik * B_k (and
// beta * Add_i) in shared memory, then the epilogue applies the drop rule, writes the row
// sorted by column, and records the row's diagonal value and sum of squares for the FP64
// traces of the next SP2 iteration.  No floating-point atomics: every output entry sums
// its terms in a fixed order, so results are bitwise reproducible.
//
// First pass (one of several variants that compute the same product; the tuner or the
// caller picks one):
//  - column blocks (paths 1, 2, 4; 7 = 2 warps, compact): a row's output columns are grouped in runs of GW (16
//    for FP64, 8 in its compact form; 32 for FP32); a per-row group table in shared memory maps a group to a
//    block of GW accumulator slots (claimed on first touch), so column j sits in bank
//    j mod 32.  R warps share a row and split each source row's entries, with a named
//    barrier between source rows.
//  - two-step (path 3; 8 = compact): one warp per row, two source rows per pass.
//  - hash (paths 10..12): a per-warp open-addressing table of 2^path slots.
// Rows whose groups outgrow the table are deferred to a one-warp 2^14-slot hash table
// (bin 1), and rows beyond that to a dense global-memory row per CTA (bin 2), so no row
// size fails.
#include <limits.h>
#include <math.h>

#include <type_traits>

#include "spgemm_internal.cuh"

namespace sp2 {

constexpr int kEmpty = -1;
// Rows of A with more entries than this skip the one-warp first pass (spgemm_super_kernel)
// and go straight to the deferred-row bins, whose one CTA per row suits their work
// (hundreds of source rows per output row, which one warp would carry alone when they fit
// its blocks).  The passes with several warps per row keep them: there, rows that fit the
// blocks finish faster than in the bins, several rows per SM at a time.
constexpr int kHeavyRowA = 512;


__device__ __forceinline__ double absval(double x) { return fabs(x); }
__device__ __forceinline__ float absval(float x) { return fabsf(x); }


// Slot layout: columns are taken in groups of 32 (j >> 5).  A group g owns the aligned
// block base(g) = 32 * h1(g) and column j first tries slot base(g) + (j & 31), so the
// first probe of column j always falls in shared-memory bank j mod 32: 32 lanes holding
// 32 different values of j mod 32 (any run of consecutive columns) never conflict.  A
// collision moves the key by an odd, group-dependent stride (double hashing), which
// visits every slot of the power-of-two table and keeps colliding groups from forming
// long primary clusters.
template <int LOG2T>
__device__ __forceinline__ int hslot0(int j) {
  const unsigned g = (unsigned)j >> 5;
  const unsigned blk = (g * 0x9E3779B1u) >> (32 - (LOG2T - 5));
  return (int)((blk << 5) | ((unsigned)j & 31u));
}
template <int LOG2T>
__device__ __forceinline__ int hstride(int j) {
  const unsigned g = (unsigned)j >> 5;
  return (int)((((g * 0x85EBCA6Bu) >> (32 - (LOG2T - 1))) << 1) | 1u);
}

// Slot holding column j, inserting it (value 0) if absent; -1 if the table is full.
template <int LOG2T, typename T>
__device__ __forceinline__ int find_or_insert(int *keys, T *vals, int j, int &ins) {
  constexpr int TS = 1 << LOG2T;
  int h = hslot0<LOG2T>(j);
  const int step = hstride<LOG2T>(j);
#pragma unroll 1
  for (int p = 0; p < TS; ++p) {
    const int cur = ((volatile int *)keys)[h];
    if (cur == j) return h;
    if (cur == kEmpty) {
      const int old = atomicCAS(keys + h, kEmpty, j);
      if (old == kEmpty) {
        vals[h] = T(0);
        ++ins;
        return h;
      }
      if (old == j) return h;
    }
    h = (h + step) & (TS - 1);
  }
  return -1;
}

template <typename T, int QM>
__device__ __forceinline__ void load_brow(const EllView<T> &B, int k, int st, int nb, int lane, int (&jr)[QM],
                                          T (&vr)[QM]) {
  const int *bi = B.idx + (size_t)k * B.w + st;
  const T *bv = B.val + (size_t)k * B.w + st;
#pragma unroll
  for (int u = 0; u < QM; ++u) {
    const int q = lane + 32 * u;
    if (q < nb) {
      jr[u] = __ldg(bi + q);
      vr[u] = __ldg(bv + q);
    } else {
      jr[u] = kEmpty;
      vr[u] = T(0);
    }
  }
}


template <typename T>
__device__ __forceinline__ bool keep_value(T v, T tau) {
  return tau == T(0) || mag_bits(v) > mag_bits(tau);
}

// In-place compaction of the occupied, kept slots to the front of the table; returns
// the kept count.
template <typename T, int TS>
__device__ __forceinline__ int compact_table(int *keys, T *vals, T tau, int lane) {
  const unsigned lt = lanemask_lt();
  const auto tb = mag_bits(tau);
  const bool keep_all = tau == T(0);
  int nk = 0;
  for (int c = 0; c < TS; c += 32) {
    const int key = keys[c + lane];
    const T v = vals[c + lane];
    const bool keep = key != kEmpty && (keep_all || mag_bits(v) > tb);
    const unsigned m = __ballot_sync(kFull, keep);
    __syncwarp();
    if (keep) {
      const int pos = nk + __popc(m & lt);
      keys[pos] = key;
      vals[pos] = v;
    }
    nk += __popc(m);
  }
  __syncwarp();
  return nk;
}

// Bitonic sort of (keys, vals)[0..nk) by key inside the warp's table (capacity >= P).
template <typename T>
__device__ __forceinline__ void sort_prefix(int *keys, T *vals, int nk, int lane) {
  int P = 32;
  while (P < nk) P <<= 1;
  for (int s = nk + lane; s < P; s += 32) keys[s] = INT_MAX;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int e = lane; e < (P >> 1); e += 32) {
        const int i = ((e & ~(j - 1)) << 1) | (e & (j - 1));
        const int ixj = i + j;
        const int ki = keys[i], kj = keys[ixj];
        const bool up = (i & k) == 0;
        if ((ki > kj) == up) {
          keys[i] = kj;
          keys[ixj] = ki;
          const T t = vals[i];
          vals[i] = vals[ixj];
          vals[ixj] = t;
        }
      }
      __syncwarp();
    }
  }
}


// Table geometry: 2^LOG2T slots of (int key, T value) per warp; a row is deferred to a
// larger table once more than LIMIT = 7/8 of the slots hold keys.  As many warps per
// CTA as fit in 224 KB of shared memory (at most 16).
template <typename T, int LOG2T>
struct HashCfg {
  static constexpr int TS = 1 << LOG2T;
  static constexpr int LIMIT = TS - TS / 8;
  static constexpr int BYTES_PER_WARP = TS * (int)(sizeof(int) + sizeof(T));
  static constexpr int WARPS_RAW = (232192 / BYTES_PER_WARP);
  static constexpr int WARPS = WARPS_RAW > 16 ? 16 : (WARPS_RAW < 1 ? 1 : WARPS_RAW);
  static constexpr int SMEM = WARPS * BYTES_PER_WARP;
};

template <typename T, int LOG2T, int QM>
__global__ void __launch_bounds__(HashCfg<T, LOG2T>::WARPS * 32, 1)
    spgemm_hash_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                       int use_add, BatchView bv, Upper up, double2 *__restrict__ rowstat, SpgemmCtl *__restrict__ ctl,
                       const int *__restrict__ row_list, const int *__restrict__ row_count,
                       int *__restrict__ fb_list, int *__restrict__ fb_count) {
  using Cfg = HashCfg<T, LOG2T>;
  constexpr int TS = Cfg::TS;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int *keys = reinterpret_cast<int *>(smem + (size_t)wid * Cfg::BYTES_PER_WARP);
  T *vals = reinterpret_cast<T *>(keys + TS);
  const int nw = gridDim.x * Cfg::WARPS;
  const int ncol = Out.n;
  // rows: all of them, or the list left by a smaller-table pass (count on the device)
  const int nrows = row_list ? *((volatile const int *)row_count) : A.n;
  int wmax = 0, wover = 0;

  for (int q = blockIdx.x * Cfg::WARPS + wid; q < nrows; q += nw) {
    const int r = row_list ? row_list[q] : q;
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (bv.row_mat) {
      const int m = bv.row_mat[r];
      if (!bv.active[m]) continue;
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    for (int s = lane * 4; s < TS; s += 128) *reinterpret_cast<int4 *>(keys + s) = make_int4(-1, -1, -1, -1);
    __syncwarp();
    int ins = 0;
    int bad = 0;
    if (add_r) {
      const int nc = min(Add.nnz[r], Add.w);
      const int d0 = up.tpd ? min(max(up.tpd[r], 0), nc) : 0;  // upper-triangle mode: from column r on
      for (int s = d0 + lane; s < nc; s += 32) {
        const int j = Add.idx[(size_t)r * Add.w + s];
        if ((unsigned)j >= (unsigned)ncol) continue;  // invalid column: ignored, never dereferenced
        const T c = Add.val[(size_t)r * Add.w + s];
        const int h = find_or_insert<LOG2T>(keys, vals, j, ins);
        if (h >= 0) vals[h] = beta_r * c; else bad = 1;
      }
      __syncwarp();
    }
    bool aborted = __reduce_add_sync(kFull, ins + (bad << 20)) > Cfg::LIMIT;

    const int na = min(A.nnz[r], A.w);
    const int *ai = A.idx + (size_t)r * A.w;
    const T *avp = A.val + (size_t)r * A.w;
    for (int base = 0; base < na && !aborted; base += 32) {
      const int s = base + lane;
      int kk = 0, nbk = 0, sk = 0;
      T av = T(0);
      if (s < na) {
        kk = __ldg(ai + s);
        if ((unsigned)kk < (unsigned)B.n) {
          av = alpha_r * __ldg(avp + s);
          nbk = min(__ldg(B.nnz + kk), B.w);
          if (up.tp) sk = min(max(__ldg(up.tp + (size_t)r * A.w + s), 0), nbk);
          nbk -= sk;
        } else {
          kk = 0;  // invalid column of A: contributes nothing
        }
      }
      const int cnt = min(32, na - base);
      int jr[QM];
      T vr[QM];
      load_brow<T, QM>(B, __shfl_sync(kFull, kk, 0), __shfl_sync(kFull, sk, 0), __shfl_sync(kFull, nbk, 0), lane,
                       jr, vr);
      for (int t = 0; t < cnt; ++t) {
        const T a = __shfl_sync(kFull, av, t);
        const int k = __shfl_sync(kFull, kk, t);
        const int st = __shfl_sync(kFull, sk, t);
        const int nb = __shfl_sync(kFull, nbk, t);
        const int nu = (nb + 31) >> 5;  // warp-uniform: register slots in use this step
        const int tn = t + 1 < cnt ? t + 1 : t;
        const int k1 = __shfl_sync(kFull, kk, tn);
        const int st1 = __shfl_sync(kFull, sk, tn);
        const int nb1 = (t + 1 < cnt) ? __shfl_sync(kFull, nbk, tn) : 0;
        int jn[QM];
        T vn[QM];
        load_brow<T, QM>(B, k1, st1, nb1, lane, jn, vn);
        // The QM columns a lane holds in this step are distinct, so their slots are too.
        // Phase 1 probes every home slot; phase 2 accumulates the hits (loads first,
        // then FMAs and stores: QM independent chains); phase 3 resolves the misses
        // (inserts, displaced keys) of all slots in one loop instead of one per slot.
        int hs[QM];
        unsigned miss = 0;
#pragma unroll
        for (int u = 0; u < QM; ++u) {
          hs[u] = -1;
          if (u < nu) {
            const bool valid = (unsigned)jr[u] < (unsigned)ncol;
            const int h = hslot0<LOG2T>(jr[u]);
            const int cur = valid ? (int)((volatile int *)keys)[h] : (int)kEmpty;
            if (valid && cur == jr[u]) hs[u] = h;
            if (valid && cur != jr[u]) miss |= 1u << u;
          }
        }
        T old[QM];
#pragma unroll
        for (int u = 0; u < QM; ++u)
          if (u < nu) old[u] = hs[u] >= 0 ? vals[hs[u]] : T(0);
#pragma unroll
        for (int u = 0; u < QM; ++u)
          if (u < nu && hs[u] >= 0) vals[hs[u]] = fmadd(a, vr[u], old[u]);
        while (miss) {
          const int u = __ffs(miss) - 1;
          miss &= miss - 1;
          int jj = jr[0];
          T vv = vr[0];
#pragma unroll
          for (int w = 1; w < QM; ++w)
            if (u == w) { jj = jr[w]; vv = vr[w]; }
          const int h = find_or_insert<LOG2T>(keys, vals, jj, ins);
          if (h >= 0) vals[h] = fmadd(a, vv, vals[h]); else bad = 1;
        }
        for (int q = lane + 32 * QM; q < nb; q += 32) {  // rows longer than 32*QM
          const int j = __ldg(B.idx + (size_t)k * B.w + st + q);
          if ((unsigned)j >= (unsigned)ncol) continue;
          const T v = __ldg(B.val + (size_t)k * B.w + st + q);
          const int h = find_or_insert<LOG2T>(keys, vals, j, ins);
          if (h >= 0) vals[h] = fmadd(a, v, vals[h]); else bad = 1;
        }
        __syncwarp();
        if (__reduce_add_sync(kFull, ins + (bad << 20)) > Cfg::LIMIT) {
          aborted = true;
          break;
        }
#pragma unroll
        for (int u = 0; u < QM; ++u) {
          jr[u] = jn[u];
          vr[u] = vn[u];
        }
      }
    }
    if (aborted) {
      if (lane == 0) {
        const int p = atomicAdd(fb_count, 1);
        fb_list[p] = r;
      }
      continue;
    }
    const int nk = compact_table<T, TS>(keys, vals, tau, lane);
    wmax = max(wmax, nk);
    if (nk > Out.w) {
      ++wover;
      if (lane == 0) rowstat[r] = make_double2(0.0, 0.0);
      continue;
    }
    sort_prefix<T>(keys, vals, nk, lane);
    int *oi = Out.idx + (size_t)r * Out.w;
    T *ov = Out.val + (size_t)r * Out.w;
    double dsum = 0.0, fsum = 0.0;
    for (int s = lane; s < nk; s += 32) {
      const int key = keys[s];
      const T v = vals[s];
      oi[s] = key;
      ov[s] = v;
      const double dv = (double)v;
      if (key == r) dsum += dv;
      fsum = fma(dv, dv, fsum);
    }
    dsum = warp_sum(dsum);
    fsum = warp_sum(fsum);
    if (lane == 0) {
      Out.nnz[r] = nk;
      rowstat[r] = make_double2(dsum, fsum);
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (wmax) atomicMax(&ctl->max_count, wmax);
    if (wover) atomicAdd(&ctl->overflow_rows, wover);
  }
}

// ------------------------------------------------------------------ block accumulator
// First pass of the multiply.  Columns are taken in groups of GW = 2^GSH consecutive
// indices.  Each group a row touches gets a dense block of GW accumulators in shared
// memory; a small open-addressing table maps group -> block (entry = g << 8 | b).  The
// accumulator of column j is vals[b * GW + (j & (GW-1))]: no per-column key, no probing,
// and the bank of a column is fixed by its low bits, so a warp holding a run of
// consecutive columns touches distinct banks.
// A row is processed by a group of R warps sharing one accumulator.  In each k step the
// columns of B_k are distinct, so the R*32 lanes split B_k's entries and update distinct
// accumulators; one barrier of the R warps orders consecutive steps (no atomics on
// values).  Blocks are cleared when the row starts (to 0, or to a signalling-NaN
// sentinel when tau == 0 so that "structural" can be told from "zero"), so handing out
// a block is a single CAS on the table.  The row comes out sorted by walking the groups
// in ascending order: no sort of the entries is needed.
// SZ = 0: blocks for a full product row; SZ = 1 (compact): about half as many, for the
// upper-triangle rows of symmetric products, so that more rows fit on an SM.
template <typename T, int SZ = 0> struct BlockCfg;
template <> struct BlockCfg<double, 0> {
  static constexpr int GSH = 4, NB = 224, LOG2G = 10;
};
template <> struct BlockCfg<float, 0> {
  static constexpr int GSH = 5, NB = 128, LOG2G = 9;
};
template <> struct BlockCfg<double, 1> {  // 8-column blocks: less of each block left unused
  static constexpr int GSH = 3, NB = 224, LOG2G = 9;
};
template <> struct BlockCfg<float, 1> {
  static constexpr int GSH = 5, NB = 80, LOG2G = 8;
};
// SZ = 2: between the two, for the denser products of converging SP2 iterations
template <> struct BlockCfg<double, 2> {
  static constexpr int GSH = 3, NB = 256, LOG2G = 9;
};
template <> struct BlockCfg<float, 2> {
  static constexpr int GSH = 5, NB = 112, LOG2G = 9;
};
template <typename T, int R, int SZ = 0>
struct BlockGeo {
  static constexpr int GSH = BlockCfg<T, SZ>::GSH, GW = 1 << GSH, NB = BlockCfg<T, SZ>::NB;
  static constexpr int LOG2G = BlockCfg<T, SZ>::LOG2G;
  static constexpr int G = 1 << LOG2G;
  static constexpr int VAL_BYTES = NB * GW * (int)sizeof(T);
  static constexpr int BYTES_PER_GROUP = VAL_BYTES + G * 4 + 16;
  static constexpr int GROUPS_RAW = 232192 / BYTES_PER_GROUP;
  // at most 32 warps per CTA (1024 threads)
  static constexpr int GROUPS_MAX0 = (SZ ? (sizeof(T) == 4 ? 20 : 32) : (sizeof(T) == 4 ? 12 : 16)) / (R > 2 ? 2 : 1);
  // R > 1: group g synchronises on named barrier g + 1, and PTX names barriers 0..15 only
  static constexpr int GROUPS_CAP = R == 1 ? 32 : (32 / R < 15 ? 32 / R : 15);
  static constexpr int GROUPS_MAX = GROUPS_MAX0 < GROUPS_CAP ? GROUPS_MAX0 : GROUPS_CAP;
  static constexpr int GROUPS = GROUPS_RAW > GROUPS_MAX ? GROUPS_MAX : (GROUPS_RAW < 1 ? 1 : GROUPS_RAW);
  static_assert(R == 1 || GROUPS <= 15, "named barriers 1..15 only");
  static constexpr int WARPS = GROUPS * R;
  static constexpr int SMEM = GROUPS * BYTES_PER_GROUP;
  // g < 2^24 - 1 fits the packed entry and never matches the empty entry 0xFFFFFFFF
  static constexpr unsigned MAX_GROUP = (1u << 24) - 1u;
};


template <int LOG2G>
__device__ __forceinline__ int ghash(unsigned g) { return (int)((g * 0x9E3779B1u) >> (32 - LOG2G)); }

// Group -> block, taking a fresh (pre-cleared) block when the group is new.  Lanes of
// different warps may race for the same group: the CAS keeps the first block, the other
// one stays unused.  Returns -1 when the blocks are used up.
template <typename T, int R, int SZ = 0>
__device__ __forceinline__ int group_block(unsigned *gtab, int *nblk, unsigned g) {
  using Geo = BlockGeo<T, R, SZ>;
  int h = ghash<Geo::LOG2G>(g);
#pragma unroll 1
  for (int p = 0; p < Geo::G; ++p) {
    const unsigned e = ((volatile unsigned *)gtab)[h];
    if ((e >> 8) == g) return (int)(e & 0xFFu);
    if (e == 0xFFFFFFFFu) {
      const int b = atomicAdd(nblk, 1);
      if (b >= Geo::NB) return -1;
      const unsigned old = atomicCAS(gtab + h, 0xFFFFFFFFu, (g << 8) | (unsigned)b);
      if (old == 0xFFFFFFFFu) return b;
      if ((old >> 8) == g) return (int)(old & 0xFFu);
    }
    h = (h + 1) & (Geo::G - 1);
  }
  return -1;
}

// Sorts the ng used entries at the front of a group table ascending (by group: the group
// sits in the high bits, distinct per entry).  One warp: in registers for ng <= 256 (REGS),
// else a bitonic network in the table itself, padded to a power of two (ng <= the table size).
template <int E>
__device__ __forceinline__ void sort_table_regs(unsigned *tab, int ng, int lane) {
  unsigned a[E];
#pragma unroll
  for (int t = 0; t < E; ++t) a[t] = lane * E + t < ng ? tab[lane * E + t] : 0xFFFFFFFFu;
  warp_bitonic<unsigned, E>(a, lane);
  __syncwarp();  // every entry is read before any is overwritten
#pragma unroll
  for (int t = 0; t < E; ++t)
    if (lane * E + t < ng) tab[lane * E + t] = a[t];
  __syncwarp();
}
// REGS = false: always the in-table network (smaller code: the multi-warp block kernel
// measured faster without the unrolled register networks; the one-warp kernel with them).
template <bool REGS>
__device__ __forceinline__ void sort_group_table(unsigned *tab, int ng, int lane) {
  __syncwarp();  // the entries were just written by other lanes
  if (ng <= 1) return;
  if (REGS) {
    if (ng <= 32) { sort_table_regs<1>(tab, ng, lane); return; }
    if (ng <= 64) { sort_table_regs<2>(tab, ng, lane); return; }
    if (ng <= 128) { sort_table_regs<4>(tab, ng, lane); return; }
    if (ng <= 256) { sort_table_regs<8>(tab, ng, lane); return; }
  }
  int P = 32;
  while (P < ng) P <<= 1;
  for (int s2 = ng + lane; s2 < P; s2 += 32) tab[s2] = 0xFFFFFFFFu;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int e = lane; e < (P >> 1); e += 32) {
        const int i = ((e & ~(jj - 1)) << 1) | (e & (jj - 1));
        const unsigned x = tab[i], y = tab[i + jj];
        if ((x > y) == ((i & k) == 0)) { tab[i] = y; tab[i + jj] = x; }
      }
      __syncwarp();
    }
}

// Barrier of the R warps of a row group (named barrier grp + 1; the warp itself when
// R == 1).  group_sync_or also returns the OR of `pred` over the group's threads, taken
// by the barrier instruction itself, so every warp sees the same value.
template <int R>
__device__ __forceinline__ void group_sync(int grp) {
  if (R == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(R * 32) : "memory");
  }
}
template <int R>
__device__ __forceinline__ bool group_sync_or(int grp, bool pred) {
  if (R == 1) {
    __syncwarp();
    return __any_sync(0xffffffffu, pred);
  }
  unsigned out;
  asm volatile(
      "{\n\t.reg .pred q, p;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"((unsigned)pred), "r"(grp + 1), "r"(R * 32)
      : "memory");
  return out != 0;
}

template <typename T, int R, int QW, bool KEEPZ, int SZ>
__global__ void __launch_bounds__(BlockGeo<T, R, SZ>::WARPS * 32, 1)
    spgemm_block_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                        int use_add, BatchView bv, Upper up, double2 *__restrict__ rowstat, SpgemmCtl *__restrict__ ctl,
                        int *__restrict__ fb_list, int *__restrict__ fb_count, unsigned char *__restrict__ route,
                        PassRows rows) {
  using Geo = BlockGeo<T, R, SZ>;
  constexpr int GW = Geo::GW, GSH = Geo::GSH, G = Geo::G;
  constexpr int SPAN = 32 * R;  // entries of a B row covered by one register slot of the group
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = wid / R, wr = wid % R, gt = wr * 32 + lane;  // group, warp in group, thread in group
  unsigned char *base = smem + (size_t)grp * Geo::BYTES_PER_GROUP;
  T *vals = reinterpret_cast<T *>(base);
  unsigned *gtab = reinterpret_cast<unsigned *>(base + Geo::VAL_BYTES);
  int *nblk = reinterpret_cast<int *>(base + Geo::VAL_BYTES + G * 4);
  const int ncol = Out.n;
  const unsigned lt = lanemask_lt();
  int wmax = 0, wover = 0;

  const int nrows = rows.list ? *rows.count : A.n;
  for (int q = blockIdx.x * Geo::GROUPS + grp; q < nrows; q += gridDim.x * Geo::GROUPS) {
    const int r = rows.list ? rows.list[q] : q;
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (bv.row_mat) {  // same row for the whole group: every warp takes the same branch
      const int m = bv.row_mat[r];
      if (!bv.active[m]) continue;
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    // flagged by an earlier product above this pass's level (it outgrew these blocks
    // there): passed on unstarted.  Every warp of the group reads the flag before the
    // barrier below, and only this group writes it, after that barrier, so the group
    // takes one branch.
    if (route && route[r] > rows.level) {
      if (gt == 0) {
        fb_list[atomicAdd(fb_count, 1)] = r;
        if (!rows.list) atomicAdd(&ctl->n_routed, 1);
      }
      continue;
    }
    {  // clear the blocks and the table
      const T c = KEEPZ ? untouched<T>() : T(0);
      constexpr int PER16 = 16 / (int)sizeof(T);
      for (int i = gt * PER16; i < Geo::NB * GW; i += SPAN * PER16) {
#pragma unroll
        for (int t = 0; t < PER16; ++t) vals[i + t] = c;
      }
      for (int i = gt * 4; i < G; i += SPAN * 4)
        *reinterpret_cast<uint4 *>(gtab + i) = make_uint4(~0u, ~0u, ~0u, ~0u);
      if (gt == 0) *nblk = 0;
    }
    group_sync<R>(grp);
    bool aborted = false;

    // Step = accumulate a * (one source row) into the blocks: first the row of the
    // addend C (a = beta), then row k of B for each entry a_ik of A's row (a = alpha*a_ik).
    // A's entries and nnz(B_k) are loaded 32 steps at a time, one chunk ahead; each warp
    // loads its share of a B row into registers two steps before it is consumed (three
    // buffers rotate).
    const int na = min(A.nnz[r], A.w);
    const int *arow_i = A.idx + (size_t)r * A.w;
    const T *arow_v = A.val + (size_t)r * A.w;
    // per entry of A: source row k, its first position read (upper-triangle mode: the
    // first column >= r, else 0) and the count of entries read from there
    int ck, cnb, nk_, nnb, cst, nst;
    T ca, na_;
    auto load_chunk = [&](int cb, int &kk, int &nbk, T &av, int &st) {
      const int s = cb + lane;
      kk = 0; nbk = 0; av = T(0); st = 0;
      if (s < na) {
        const int k = __ldg(arow_i + s);
        if ((unsigned)k < (unsigned)B.n) {
          kk = k;
          av = alpha_r * __ldg(arow_v + s);
          nbk = min(__ldg(B.nnz + k), B.w);
          if (up.tp) st = min(max(__ldg(up.tp + (size_t)r * A.w + s), 0), nbk);
          nbk -= st;
        }
      }
    };
    load_chunk(0, ck, cnb, ca, cst);
    load_chunk(32, nk_, nnb, na_, nst);
    int cbase = 0;
    auto info = [&](int t, int &k, int &nb, T &a, int &st) {  // t in [cbase, cbase + 64)
      if (t < cbase + 32) {
        k = __shfl_sync(kFull, ck, t & 31);
        nb = __shfl_sync(kFull, cnb, t & 31);
        a = __shfl_sync(kFull, ca, t & 31);
        st = __shfl_sync(kFull, cst, t & 31);
      } else {
        k = __shfl_sync(kFull, nk_, t & 31);
        nb = __shfl_sync(kFull, nnb, t & 31);
        a = __shfl_sync(kFull, na_, t & 31);
        st = __shfl_sync(kFull, nst, t & 31);
      }
    };
    auto fetch = [&](const int *ri, const T *rv, int nb, int (&jr)[QW], T (&vr)[QW]) {
#pragma unroll
      for (int u = 0; u < QW; ++u) {
        const int q = SPAN * u + gt;
        jr[u] = q < nb ? __ldg(ri + q) : -1;
        vr[u] = q < nb ? __ldg(rv + q) : T(0);
      }
    };
    auto fetch_step = [&](int t, int (&jr)[QW], T (&vr)[QW], int &nb, T &a, size_t &off) {
      int k, st;
      info(t, k, nb, a, st);
      off = (size_t)k * B.w + st;
      fetch(B.idx + off, B.val + off, nb, jr, vr);
    };
    // accumulate one step from registers, body instantiated per number NU of occupied
    // register slots of this warp (warp-uniform switch: empty slots cost nothing)
    auto step_nu = [&](auto nu_c, const int (&jr)[QW], const T (&vr)[QW], T a, const unsigned (&hint)[QW]) {
      constexpr int NU = decltype(nu_c)::value;
      int sl[NU];
      unsigned miss = 0;
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        sl[u] = -1;
        const unsigned g = (unsigned)jr[u] >> GSH;
        if ((unsigned)jr[u] < (unsigned)ncol) {
          // the entry read before the last barrier, if it already holds g (entries are
          // never changed once set), else a fresh read
          unsigned e = hint[u];
          if ((e >> 8) != g) e = ((volatile unsigned *)gtab)[ghash<Geo::LOG2G>(g)];
          if ((e >> 8) == g) sl[u] = (int)(e & 0xFFu) * GW + (jr[u] & (GW - 1));
          else miss |= 1u << u;
        }
      }
      // misses: one elected lane per distinct group of this warp finds or takes a block
      while (__any_sync(kFull, miss != 0)) {
        const int u = miss ? __ffs(miss) - 1 : -1;
        int jj = jr[0];
#pragma unroll
        for (int w = 1; w < NU; ++w)
          if (u == w) jj = jr[w];
        const unsigned act = __ballot_sync(kFull, u >= 0);
        if (u >= 0) {
          const unsigned g = (unsigned)jj >> GSH;
          const unsigned peers = __match_any_sync(act, g);
          const int leader = __ffs(peers) - 1;
          int b = -1;
          if (lane == leader) b = g < Geo::MAX_GROUP ? group_block<T, R, SZ>(gtab, nblk, g) : -1;
          b = __shfl_sync(peers, b, leader);
#pragma unroll
          for (int w = 0; w < NU; ++w)
            if (u == w) sl[w] = b < 0 ? -1 : b * GW + (jj & (GW - 1));
          if (b < 0) aborted = true;
          miss &= miss - 1;
        }
      }
      T old[NU];
#pragma unroll
      for (int u = 0; u < NU; ++u) old[u] = sl[u] >= 0 ? vals[sl[u]] : T(0);
#pragma unroll
      for (int u = 0; u < NU; ++u)
        if (sl[u] >= 0) {
          const T o = (KEEPZ && is_untouched(old[u])) ? T(0) : old[u];
          vals[sl[u]] = fmadd(a, vr[u], o);
        }
    };
    // hints: the table entries at the first probe of the next step's register slots, read
    // before this step's barrier so that their latency overlaps it
    unsigned hint[QW];
#pragma unroll
    for (int u = 0; u < QW; ++u) hint[u] = 0xFFFFFFFFu;
    auto step = [&](const int (&jr)[QW], const T (&vr)[QW], int nb, T a, const int *ri, const T *rv,
                    const int (&jn)[QW]) {
      const int mine = nb > 32 * wr ? (nb - 32 * wr + SPAN - 1) / SPAN : 0;  // slots of this warp
      const int nu = min(mine, QW);
      switch (nu) {
        case 0: break;
        case 1: step_nu(std::integral_constant<int, 1>{}, jr, vr, a, hint); break;
        case 2: step_nu(std::integral_constant<int, (QW >= 2 ? 2 : QW)>{}, jr, vr, a, hint); break;
        case 3: step_nu(std::integral_constant<int, (QW >= 3 ? 3 : QW)>{}, jr, vr, a, hint); break;
        case 4: step_nu(std::integral_constant<int, (QW >= 4 ? 4 : QW)>{}, jr, vr, a, hint); break;
        case 5: step_nu(std::integral_constant<int, (QW >= 5 ? 5 : QW)>{}, jr, vr, a, hint); break;
        case 6: step_nu(std::integral_constant<int, (QW >= 6 ? 6 : QW)>{}, jr, vr, a, hint); break;
        case 7: step_nu(std::integral_constant<int, (QW >= 7 ? 7 : QW)>{}, jr, vr, a, hint); break;
        default: step_nu(std::integral_constant<int, QW>{}, jr, vr, a, hint); break;
      }
      if (nb > SPAN * QW) {  // rows longer than the registers: same phases, from memory
        unsigned none[QW];
#pragma unroll
        for (int u = 0; u < QW; ++u) none[u] = 0xFFFFFFFFu;
        for (int q0 = SPAN * QW; q0 < nb; q0 += SPAN) {
          const int q = q0 + gt;
          int jt[QW];
          T vt[QW];
          jt[0] = q < nb ? __ldg(ri + q) : -1;
          vt[0] = q < nb ? __ldg(rv + q) : T(0);
          step_nu(std::integral_constant<int, 1>{}, jt, vt, a, none);
        }
      }
#pragma unroll
      for (int u = 0; u < QW; ++u)
        hint[u] = (unsigned)jn[u] < (unsigned)ncol
                      ? ((volatile unsigned *)gtab)[ghash<Geo::LOG2G>((unsigned)jn[u] >> GSH)]
                      : 0xFFFFFFFFu;
      aborted = group_sync_or<R>(grp, aborted);  // orders this step's updates before the next step's
    };

    int j0[QW], j1[QW], j2[QW];
    T v0[QW], v1[QW], v2[QW];
    int nb0 = 0, nb1 = 0, nb2 = 0;
    size_t k0 = 0, k1 = 0, k2 = 0;  // offsets of the source rows in B's arrays
    T a0 = T(0), a1 = T(0), a2 = T(0);
    if (add_r) {
      int nc = min(Add.nnz[r], Add.w);
      const int d0 = up.tpd ? min(max(up.tpd[r], 0), nc) : 0;
      const int *ci = Add.idx + (size_t)r * Add.w + d0;
      const T *cv = Add.val + (size_t)r * Add.w + d0;
      nc -= d0;
      fetch(ci, cv, nc, j2, v2);
      if (na > 0) fetch_step(0, j0, v0, nb0, a0, k0);
      if (na > 1) fetch_step(1, j1, v1, nb1, a1, k1);
      step(j2, v2, nc, beta_r, ci, cv, j0);
    } else {
      if (na > 0) fetch_step(0, j0, v0, nb0, a0, k0);
      if (na > 1) fetch_step(1, j1, v1, nb1, a1, k1);
    }
    for (int t = 0; t < na && !aborted; t += 3) {
      if (t >= cbase + 32) {  // next chunk of A's entries becomes current
        ck = nk_; cnb = nnb; ca = na_; cst = nst;
        cbase += 32;
        load_chunk(cbase + 32, nk_, nnb, na_, nst);
      }
      if (t + 2 < na) fetch_step(t + 2, j2, v2, nb2, a2, k2);
      step(j0, v0, nb0, a0, B.idx + k0, B.val + k0, j1);
      if (t + 1 >= na || aborted) break;
      if (t + 3 < na) fetch_step(t + 3, j0, v0, nb0, a0, k0);
      step(j1, v1, nb1, a1, B.idx + k1, B.val + k1, j2);
      if (t + 2 >= na || aborted) break;
      if (t + 4 < na) fetch_step(t + 4, j1, v1, nb1, a1, k1);
      step(j2, v2, nb2, a2, B.idx + k2, B.val + k2, j0);
    }
    if (aborted) {
      if (gt == 0) {
        const int p = atomicAdd(fb_count, 1);
        fb_list[p] = r;
        if (route) route[r] = (unsigned char)(rows.level + 1);
      }
      group_sync<R>(grp);
      continue;
    }
    if (wr == 0) {
      // compact the used group entries to the front of the table, sort them by group
      int ng = 0;
      for (int c = 0; c < G; c += 32) {
        const unsigned e = gtab[c + lane];
        const bool used = e != 0xFFFFFFFFu;
        const unsigned m = __ballot_sync(kFull, used);
        __syncwarp();
        if (used) gtab[ng + __popc(m & lt)] = e;
        ng += __popc(m);
      }
      sort_group_table<false>(gtab, ng, lane);
      // walk the groups in column order: 32 / GW groups per pass, lane -> column
      const auto tb = mag_bits(tau);
      int nk = 0;
      double dsum = 0.0, fsum = 0.0;
      int *oi = Out.idx + (size_t)r * Out.w;
      T *ov = Out.val + (size_t)r * Out.w;
      constexpr int GPP = 32 / GW;
      for (int c = 0; c < ng; c += GPP) {
        const int gi = c + lane / GW;
        bool keep = false;
        int j = 0;
        T v = T(0);
        if (gi < ng) {
          const unsigned e = gtab[gi];
          const int b = (int)(e & 0xFFu);
          j = (int)((e >> 8) << GSH) + (lane & (GW - 1));
          v = vals[b * GW + (lane & (GW - 1))];
          keep = KEEPZ ? !is_untouched(v) : mag_bits(v) > tb;
        }
        const unsigned m = __ballot_sync(kFull, keep);
        if (keep) {
          const int pos = nk + __popc(m & lt);
          if (pos < Out.w) { oi[pos] = j; ov[pos] = v; }
          if (!up.tp) {  // upper-triangle rows: the mirror pass takes the statistics of the full rows
            const double dv = (double)v;
            if (j == r) dsum += dv;
            fsum = fma(dv, dv, fsum);
          }
        }
        nk += __popc(m);
      }
      dsum = warp_sum(dsum);
      fsum = warp_sum(fsum);
      wmax = max(wmax, nk);
      if (lane == 0) {
        if (nk > Out.w) {
          ++wover;
          rowstat[r] = make_double2(0.0, 0.0);
        } else {
          Out.nnz[r] = nk;
          rowstat[r] = make_double2(dsum, fsum);
        }
      }
    }
    group_sync<R>(grp);  // the accumulator is free for the next row
  }
  if (lane == 0 && wr == 0) {
    if (wmax) atomicMax(&ctl->max_count, wmax);
    if (wover) atomicAdd(&ctl->overflow_rows, wover);
  }
}

// ------------------------------------------------------------------ super-step variant
// Same column-block accumulator, one warp per row, but S consecutive k steps form a
// super-step: the table lookups of all S rows of B are issued together (S*QM independent
// chains), misses are resolved once, then the S read-modify-write passes run back to
// back separated only by __syncwarp (consecutive passes may touch the same accumulator).
// Register slots are predicated instead of specialised, which keeps the code small.
template <typename T, int QM, int S, bool KEEPZ, int SZ>
__global__ void __launch_bounds__(BlockGeo<T, 1, SZ>::WARPS * 32, 1)
    spgemm_super_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                        int use_add, BatchView bv, Upper up, double2 *__restrict__ rowstat, SpgemmCtl *__restrict__ ctl,
                        int *__restrict__ fb_list, int *__restrict__ fb_count, unsigned char *__restrict__ route,
                        PassRows rows) {
  using Geo = BlockGeo<T, 1, SZ>;
  constexpr int GW = Geo::GW, GSH = Geo::GSH, G = Geo::G;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *base = smem + (size_t)wid * Geo::BYTES_PER_GROUP;
  T *vals = reinterpret_cast<T *>(base);
  unsigned *gtab = reinterpret_cast<unsigned *>(base + Geo::VAL_BYTES);
  int *nblk = reinterpret_cast<int *>(base + Geo::VAL_BYTES + G * 4);
  const int ncol = Out.n;
  const unsigned lt = lanemask_lt();
  int wmax = 0, wover = 0;

  const int nrows = rows.list ? *rows.count : A.n;
  for (int q = blockIdx.x * Geo::GROUPS + wid; q < nrows; q += gridDim.x * Geo::GROUPS) {
    const int r = rows.list ? rows.list[q] : q;
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (bv.row_mat) {
      const int m = bv.row_mat[r];
      if (!bv.active[m]) continue;
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    if (A.nnz[r] > kHeavyRowA) {  // straight to the deferred-row bins (see kHeavyRowA)
      if (lane == 0) {
        fb_list[atomicAdd(fb_count, 1)] = r;
        if (!rows.list) atomicAdd(&ctl->n_heavy, 1);
      }
      continue;
    }
    if (route && route[r] > rows.level) {  // flagged above this level: passed on unstarted
      if (lane == 0) {
        fb_list[atomicAdd(fb_count, 1)] = r;
        if (!rows.list) atomicAdd(&ctl->n_routed, 1);
      }
      continue;
    }
    {
      const T c = KEEPZ ? untouched<T>() : T(0);
      for (int i = lane; i < Geo::NB * GW; i += 32) vals[i] = c;
      for (int i = lane * 4; i < G; i += 128) *reinterpret_cast<uint4 *>(gtab + i) = make_uint4(~0u, ~0u, ~0u, ~0u);
      if (lane == 0) *nblk = 0;
    }
    __syncwarp();
    bool aborted = false;
    const int na = min(A.nnz[r], A.w);
    const int nc0 = add_r ? min(Add.nnz[r], Add.w) : 0;
    const int d0 = (add_r && up.tpd) ? min(max(up.tpd[r], 0), nc0) : 0;  // upper-triangle mode: from column r on
    const int nc = nc0 - d0;
    const int nsteps = na + (add_r ? 1 : 0);  // step 0 is the addend row, if any
    const int *arow_i = A.idx + (size_t)r * A.w;
    const T *arow_v = A.val + (size_t)r * A.w;
    // A's entries for 32 steps at a time (k, nnz(B_k), alpha*a_ik), next chunk preloaded
    int ck, cnb, nk_, nnb, cst, nst;
    T ca, na_;
    auto load_chunk = [&](int cb, int &kk, int &nbk, T &av, int &st) {
      const int s0 = cb + lane;
      kk = 0; nbk = 0; av = T(0); st = 0;
      if (s0 < na) {
        const int k = __ldg(arow_i + s0);
        if ((unsigned)k < (unsigned)B.n) {
          kk = k;
          av = alpha_r * __ldg(arow_v + s0);
          nbk = min(__ldg(B.nnz + k), B.w);
          if (up.tp) st = min(max(__ldg(up.tp + (size_t)r * A.w + s0), 0), nbk);
          nbk -= st;
        }
      }
    };
    load_chunk(0, ck, cnb, ca, cst);
    load_chunk(32, nk_, nnb, na_, nst);
    int cbase = 0;
    // source row of step t (t in [cbase, cbase+64) for the A part)
    auto src = [&](int t, const int *&ri, const T *&rv, int &nb, T &a) {
      if (add_r && t == 0) {
        ri = Add.idx + (size_t)r * Add.w + d0; rv = Add.val + (size_t)r * Add.w + d0; nb = nc; a = beta_r;
        return;
      }
      const int ta = t - (add_r ? 1 : 0);
      int k, st;
      if (ta < cbase + 32) {
        k = __shfl_sync(kFull, ck, ta & 31); nb = __shfl_sync(kFull, cnb, ta & 31); a = __shfl_sync(kFull, ca, ta & 31);
        st = __shfl_sync(kFull, cst, ta & 31);
      } else {
        k = __shfl_sync(kFull, nk_, ta & 31); nb = __shfl_sync(kFull, nnb, ta & 31); a = __shfl_sync(kFull, na_, ta & 31);
        st = __shfl_sync(kFull, nst, ta & 31);
      }
      ri = B.idx + (size_t)k * B.w + st; rv = B.val + (size_t)k * B.w + st;
    };
    int jc[S][QM], jn[S][QM];
    T vc[S][QM], vn[S][QM];
    int nbc[S], nbn[S];
    T ac[S], an[S];
    const int *ric[S], *rin[S];
    const T *rvc[S], *rvn[S];
    auto load_super = [&](int t0, int (&jr)[S][QM], T (&vr)[S][QM], int (&nbr)[S], T (&ar)[S], const int *(&rir)[S],
                          const T *(&rvr)[S]) {
#pragma unroll
      for (int q = 0; q < S; ++q) {
        nbr[q] = 0; ar[q] = T(0); rir[q] = B.idx; rvr[q] = B.val;
        if (t0 + q < nsteps) src(t0 + q, rir[q], rvr[q], nbr[q], ar[q]);
#pragma unroll
        for (int u = 0; u < QM; ++u) {
          const int e = 32 * u + lane;
          jr[q][u] = e < nbr[q] ? __ldg(rir[q] + e) : -1;
          vr[q][u] = e < nbr[q] ? __ldg(rvr[q] + e) : T(0);
        }
      }
    };
    load_super(0, jc, vc, nbc, ac, ric, rvc);
    for (int t0 = 0; t0 < nsteps && !aborted; t0 += S) {
      // chunk of A entries: steps t0 .. t0+2S-1 must lie in [cbase, cbase+64)
      const int ta_next = t0 + S + S - 1 - (add_r ? 1 : 0);
      if (ta_next >= cbase + 64) {
        ck = nk_; cnb = nnb; ca = na_; cst = nst;
        cbase += 32;
        load_chunk(cbase + 32, nk_, nnb, na_, nst);
      }
      load_super(t0 + S, jn, vn, nbn, an, rin, rvn);  // prefetch the next super-step
      // phase A: every held column of the S rows -> accumulator index
      int sl[S][QM];
      unsigned miss = 0;
#pragma unroll
      for (int q = 0; q < S; ++q)
#pragma unroll
        for (int u = 0; u < QM; ++u) {
          sl[q][u] = -1;
          const int j = jc[q][u];
          if ((unsigned)j < (unsigned)ncol) {
            const unsigned g = (unsigned)j >> GSH;
            const unsigned e = ((volatile unsigned *)gtab)[ghash<Geo::LOG2G>(g)];
            if ((e >> 8) == g) sl[q][u] = (int)(e & 0xFFu) * GW + (j & (GW - 1));
            else miss |= 1u << (q * QM + u);
          }
        }
      while (__any_sync(kFull, miss != 0)) {
        const int m = miss ? __ffs(miss) - 1 : -1;
        int jj = -1;
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
          for (int u = 0; u < QM; ++u)
            if (m == q * QM + u) jj = jc[q][u];
        const unsigned act = __ballot_sync(kFull, m >= 0);
        if (m >= 0) {
          const unsigned g = (unsigned)jj >> GSH;
          const unsigned peers = __match_any_sync(act, g);
          const int leader = __ffs(peers) - 1;
          int b = -1;
          if (lane == leader) b = g < Geo::MAX_GROUP ? group_block<T, 1, SZ>(gtab, nblk, g) : -1;
          b = __shfl_sync(peers, b, leader);
#pragma unroll
          for (int q = 0; q < S; ++q)
#pragma unroll
            for (int u = 0; u < QM; ++u)
              if (m == q * QM + u) sl[q][u] = b < 0 ? -1 : b * GW + (jj & (GW - 1));
          if (b < 0) aborted = true;
          miss &= miss - 1;
        }
      }
      __syncwarp();
      // phase B: one read-modify-write pass per row of the super-step
#pragma unroll
      for (int q = 0; q < S; ++q) {
        T old[QM];
#pragma unroll
        for (int u = 0; u < QM; ++u) old[u] = sl[q][u] >= 0 ? vals[sl[q][u]] : T(0);
#pragma unroll
        for (int u = 0; u < QM; ++u)
          if (sl[q][u] >= 0) {
            const T o = (KEEPZ && is_untouched(old[u])) ? T(0) : old[u];
            vals[sl[q][u]] = fmadd(ac[q], vc[q][u], o);
          }
        // entries beyond the registers (rows longer than 32*QM), from memory
        for (int e0 = 32 * QM; e0 < nbc[q]; e0 += 32) {
          const int e = e0 + lane;
          const int j = e < nbc[q] ? __ldg(ric[q] + e) : -1;
          int slt = -1;
          if ((unsigned)j < (unsigned)ncol) {
            const unsigned g = (unsigned)j >> GSH;
            const unsigned en = ((volatile unsigned *)gtab)[ghash<Geo::LOG2G>(g)];
            if ((en >> 8) == g) slt = (int)(en & 0xFFu) * GW + (j & (GW - 1));
          }
          unsigned tmiss = __ballot_sync(kFull, slt < 0 && (unsigned)j < (unsigned)ncol);
          if (tmiss & (1u << lane)) {
            const unsigned g = (unsigned)j >> GSH;
            const unsigned peers = __match_any_sync(tmiss, g);
            const int leader = __ffs(peers) - 1;
            int b = -1;
            if (lane == leader) b = g < Geo::MAX_GROUP ? group_block<T, 1, SZ>(gtab, nblk, g) : -1;
            b = __shfl_sync(peers, b, leader);
            slt = b < 0 ? -1 : b * GW + (j & (GW - 1));
            if (b < 0) aborted = true;
          }
          __syncwarp();
          if (slt >= 0) {
            const T o0 = vals[slt];
            const T o = (KEEPZ && is_untouched(o0)) ? T(0) : o0;
            vals[slt] = fmadd(ac[q], __ldg(rvc[q] + e), o);
          }
        }
        __syncwarp();
      }
      aborted = __any_sync(kFull, aborted);
#pragma unroll
      for (int q = 0; q < S; ++q) {
        nbc[q] = nbn[q]; ac[q] = an[q]; ric[q] = rin[q]; rvc[q] = rvn[q];
#pragma unroll
        for (int u = 0; u < QM; ++u) { jc[q][u] = jn[q][u]; vc[q][u] = vn[q][u]; }
      }
    }
    if (aborted) {
      if (lane == 0) {
        const int p = atomicAdd(fb_count, 1);
        fb_list[p] = r;
        if (route) route[r] = (unsigned char)(rows.level + 1);
      }
      continue;
    }
    // epilogue: groups in order, lane -> column (as in the block kernel)
    int ng = 0;
    for (int c = 0; c < G; c += 32) {
      const unsigned e = gtab[c + lane];
      const bool used = e != 0xFFFFFFFFu;
      const unsigned m = __ballot_sync(kFull, used);
      __syncwarp();
      if (used) gtab[ng + __popc(m & lt)] = e;
      ng += __popc(m);
    }
    sort_group_table<true>(gtab, ng, lane);
    const auto tb = mag_bits(tau);
    int nk = 0;
    double dsum = 0.0, fsum = 0.0;
    int *oi = Out.idx + (size_t)r * Out.w;
    T *ov = Out.val + (size_t)r * Out.w;
    constexpr int GPP = 32 / GW;
    for (int c = 0; c < ng; c += GPP) {
      const int gi = c + lane / GW;
      bool keep = false;
      int j = 0;
      T v = T(0);
      if (gi < ng) {
        const unsigned e = gtab[gi];
        const int b = (int)(e & 0xFFu);
        j = (int)((e >> 8) << GSH) + (lane & (GW - 1));
        v = vals[b * GW + (lane & (GW - 1))];
        keep = KEEPZ ? !is_untouched(v) : mag_bits(v) > tb;
      }
      const unsigned m = __ballot_sync(kFull, keep);
      if (keep) {
        const int pos = nk + __popc(m & lt);
        if (pos < Out.w) { oi[pos] = j; ov[pos] = v; }
        if (!up.tp) {  // upper-triangle rows: the mirror pass takes the statistics of the full rows
          const double dv = (double)v;
          if (j == r) dsum += dv;
          fsum = fma(dv, dv, fsum);
        }
      }
      nk += __popc(m);
    }
    dsum = warp_sum(dsum);
    fsum = warp_sum(fsum);
    wmax = max(wmax, nk);
    if (lane == 0) {
      if (nk > Out.w) {
        ++wover;
        rowstat[r] = make_double2(0.0, 0.0);
      } else {
        Out.nnz[r] = nk;
        rowstat[r] = make_double2(dsum, fsum);
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (wmax) atomicMax(&ctl->max_count, wmax);
    if (wover) atomicAdd(&ctl->overflow_rows, wover);
  }
}

// ------------------------------------------------------------------ large rows
// One CTA per deferred row: accumulate into a dense row of n values in global memory
// (per-CTA slot; marks start at -1 and accumulators at 0 and are restored after use),
// then scan the columns in ascending order, so the output comes out sorted.
constexpr int kDenseThreads = 512;

template <typename T>
__device__ __forceinline__ int block_exclusive_scan_ballot(bool flag, int *s_warp, int &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(kFull, flag);
  if (lane == 0) s_warp[wid] = __popc(m);
  __syncthreads();
  int before = 0;
  total = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    const int c = s_warp[w];
    if (w < wid) before += c;
    total += c;
  }
  const int pos = before + __popc(m & lanemask_lt());
  __syncthreads();
  return pos;
}

template <typename T>
__global__ void __launch_bounds__(kDenseThreads)
    spgemm_dense_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                        int use_add, BatchView bv, Upper up, double2 *__restrict__ rowstat, SpgemmCtl *__restrict__ ctl,
                        const int *__restrict__ fb_list, const int *__restrict__ fb_count, T *__restrict__ acc_all,
                        int *__restrict__ mark_all) {
  __shared__ int s_warp[kDenseThreads / 32];
  __shared__ double s_d[kDenseThreads / 32], s_f[kDenseThreads / 32];
  const int n = Out.n;  // columns of the product
  const int nfb = *((volatile const int *)fb_count);
  T *acc = acc_all + (size_t)blockIdx.x * n;
  int *mark = mark_all + (size_t)blockIdx.x * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int lmax = 0, lover = 0;
  for (int q = blockIdx.x; q < nfb; q += gridDim.x) {
    const int r = fb_list[q];
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (bv.row_mat) {  // deferred rows belong to active matrices
      const int m = bv.row_mat[r];
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    if (add_r) {
      const int nc = min(Add.nnz[r], Add.w);
      const int d0 = up.tpd ? min(max(up.tpd[r], 0), nc) : 0;  // upper-triangle mode: from column r on
      for (int s = d0 + threadIdx.x; s < nc; s += blockDim.x) {
        const int j = Add.idx[(size_t)r * Add.w + s];
        if ((unsigned)j >= (unsigned)n) continue;
        mark[j] = 1;
        acc[j] += beta_r * Add.val[(size_t)r * Add.w + s];
      }
    }
    __syncthreads();
    // one k at a time in A's row order: the columns of B_k are distinct, so the CTA's
    // threads update distinct accumulators; the barrier orders the steps (deterministic)
    const int na = min(A.nnz[r], A.w);
    for (int t = 0; t < na; ++t) {
      const int k = A.idx[(size_t)r * A.w + t];
      if ((unsigned)k < (unsigned)B.n) {
        const T a = alpha_r * A.val[(size_t)r * A.w + t];
        const int nb = min(B.nnz[k], B.w);
        const int st = up.tp ? min(max(up.tp[(size_t)r * A.w + t], 0), nb) : 0;
        for (int s = st + threadIdx.x; s < nb; s += blockDim.x) {
          const int j = B.idx[(size_t)k * B.w + s];
          if ((unsigned)j >= (unsigned)n) continue;
          mark[j] = 1;
          acc[j] = fmadd(a, B.val[(size_t)k * B.w + s], acc[j]);
        }
      }
      __syncthreads();
    }
    int base = 0;
    double d = 0.0, f = 0.0;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
      const int j = c0 + threadIdx.x;
      bool keep = false;
      T v = T(0);
      if (j < n && mark[j] != -1) {
        v = acc[j];
        keep = keep_value(v, tau);
        mark[j] = -1;
        acc[j] = T(0);
      }
      int total;
      const int pos = base + block_exclusive_scan_ballot<T>(keep, s_warp, total);
      if (keep) {
        if (pos < Out.w) {
          Out.idx[(size_t)r * Out.w + pos] = j;
          Out.val[(size_t)r * Out.w + pos] = v;
        }
        const double dv = (double)v;
        if (j == r) d += dv;
        f += dv * dv;
      }
      base += total;
    }
    d = warp_sum(d);
    f = warp_sum(f);
    if (lane == 0) { s_d[wid] = d; s_f[wid] = f; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double dd = 0.0, ff = 0.0;
      for (int w = 0; w < nwarp; ++w) { dd += s_d[w]; ff += s_f[w]; }
      rowstat[r] = make_double2(dd, ff);
      lmax = max(lmax, base);
      if (base > Out.w) ++lover; else Out.nnz[r] = base;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (lmax) atomicMax(&ctl->max_count, lmax);
    if (lover) atomicAdd(&ctl->overflow_rows, lover);
  }
}

// ------------------------------------------------------------------ window bin
// One CTA per deferred row whose product columns span at most WIN (banded rows: the
// paper's chain model Hamiltonians).  The row accumulates in a dense window of shared
// memory indexed by column - lo (no lookup), one source row at a time with a barrier
// between them (deterministic), a bit per column marking the structural entries; then
// the window is scanned in column order.  Rows with a wider span go on to the next bin.
constexpr int kWinThreads = 512;
constexpr int kWinPre = 8;  // entries of the next source row each thread holds in registers
template <typename T>
struct WinCfg {
  static constexpr int WIN = (192 * 1024) / (int)sizeof(T);
  static constexpr int SMEM = WIN * (int)sizeof(T) + (WIN / 32) * 4;
};

template <typename T>
__global__ void __launch_bounds__(kWinThreads)
    spgemm_window_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                         int use_add, BatchView bv, Upper up, double2 *__restrict__ rowstat, SpgemmCtl *__restrict__ ctl,
                         const int *__restrict__ in_list, const int *__restrict__ in_count, int *__restrict__ out_list,
                         int *__restrict__ out_count) {
  using Cfg = WinCfg<T>;
  extern __shared__ __align__(16) unsigned char smem[];
  T *acc = reinterpret_cast<T *>(smem);
  unsigned *touched = reinterpret_cast<unsigned *>(smem + (size_t)Cfg::WIN * sizeof(T));
  __shared__ int s_warp[kWinThreads / 32];
  __shared__ int s_lo[kWinThreads / 32], s_hi[kWinThreads / 32];
  __shared__ double s_d[kWinThreads / 32], s_f[kWinThreads / 32];
  const int ncol = Out.n;
  const int nrows = *((volatile const int *)in_count);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const auto tb = mag_bits(tau);
  // structural entries need marks only when tau = 0 (a slot nothing reached holds 0,
  // which any tau > 0 drops)
  const bool marks = tau == T(0);
  // marks of one pass: the lanes of a warp that share a mark word OR their bits and one
  // of them sets them (consecutive columns share words)
  auto mark = [&](bool on, int c) {
    const unsigned act = __ballot_sync(kFull, on);
    if (on) {
      const unsigned word = (unsigned)c >> 5;
      const unsigned peers = __match_any_sync(act, word);
      const unsigned bits = __reduce_or_sync(peers, 1u << (c & 31));
      if (lane == __ffs(peers) - 1) atomicOr(touched + word, bits);
    }
  };
  int lmax = 0, lover = 0;
  for (int q = blockIdx.x; q < nrows; q += gridDim.x) {
    const int r = in_list[q];
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (bv.row_mat) {  // deferred rows belong to active matrices
      const int m = bv.row_mat[r];
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    const int na = min(A.nnz[r], A.w);
    const int nc = add_r ? min(Add.nnz[r], Add.w) : 0;
    const int d0 = (add_r && up.tpd) ? min(max(up.tpd[r], 0), nc) : 0;
    // column span of the row: first and last column of every source row (sorted rows)
    int lo = INT_MAX, hi = -1;
    for (int t = threadIdx.x; t < na; t += blockDim.x) {
      const int k = A.idx[(size_t)r * A.w + t];
      if ((unsigned)k >= (unsigned)B.n) continue;
      const int nb = min(B.nnz[k], B.w);
      const int st = up.tp ? min(max(up.tp[(size_t)r * A.w + t], 0), nb) : 0;
      if (st < nb) {
        lo = min(lo, B.idx[(size_t)k * B.w + st]);
        hi = max(hi, B.idx[(size_t)k * B.w + nb - 1]);
      }
    }
    if (threadIdx.x == 0 && d0 < nc) {
      lo = min(lo, Add.idx[(size_t)r * Add.w + d0]);
      hi = max(hi, Add.idx[(size_t)r * Add.w + nc - 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(kFull, lo, o));
      hi = max(hi, __shfl_xor_sync(kFull, hi, o));
    }
    if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; }
    __syncthreads();
    lo = INT_MAX; hi = -1;
    for (int w = 0; w < nwarp; ++w) { lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); }
    lo = max(lo, 0);
    hi = min(hi, ncol - 1);
    __syncthreads();
    if (hi >= lo && hi - lo + 1 > Cfg::WIN) {  // too wide: the next bin
      if (threadIdx.x == 0) out_list[atomicAdd(out_count, 1)] = r;
      continue;
    }
    const int span = hi >= lo ? hi - lo + 1 : 0;
    for (int c = threadIdx.x; c < span; c += blockDim.x) acc[c] = T(0);
    if (marks)
      for (int c = threadIdx.x; c < (span + 31) / 32; c += blockDim.x) touched[c] = 0u;
    __syncthreads();
    if (d0 < nc) {
      for (int s0 = d0; s0 < nc; s0 += blockDim.x) {  // warp-uniform trip count (the marks vote)
        const int s = s0 + threadIdx.x;
        const int j = s < nc ? Add.idx[(size_t)r * Add.w + s] : -1;
        const bool in = s < nc && j >= lo && j <= hi;
        if (in) acc[j - lo] = fmadd(beta_r, Add.val[(size_t)r * Add.w + s], acc[j - lo]);
        if (marks) mark(in, j - lo);
      }
      __syncthreads();
    }
    // one source row at a time in A's row order: its columns are distinct, so threads
    // update distinct accumulators; the barrier orders the source rows
    if (marks) {
      for (int t = 0; t < na; ++t) {
        const int k = A.idx[(size_t)r * A.w + t];
        if ((unsigned)k < (unsigned)B.n) {
          const T a = alpha_r * A.val[(size_t)r * A.w + t];
          const int nb = min(B.nnz[k], B.w);
          const int st = up.tp ? min(max(up.tp[(size_t)r * A.w + t], 0), nb) : 0;
          for (int s0 = st; s0 < nb; s0 += blockDim.x) {  // warp-uniform trip count (the marks vote)
            const int s = s0 + threadIdx.x;
            const int j = s < nb ? B.idx[(size_t)k * B.w + s] : -1;
            const bool in = s < nb && j >= lo && j <= hi;
            if (in) acc[j - lo] = fmadd(a, B.val[(size_t)k * B.w + s], acc[j - lo]);
            mark(in, j - lo);
          }
        }
        __syncthreads();
      }
    } else {
      // the next source row is loaded into registers (kWinPre entries per thread) while
      // the current one accumulates, so a step waits on no global load
      int cj[kWinPre], nj[kWinPre];
      T cv[kWinPre], nv[kWinPre];
      T ca = T(0), an = T(0);
      const int *crow = B.idx;
      const T *cvrow = B.val;
      int cnb = 0, cst = 0, nnb = 0, nst = 0;
      const int *nrow = B.idx;
      const T *nvrow = B.val;
      auto fetch = [&](int t, int (&jr)[kWinPre], T (&vr)[kWinPre], T &a, const int *&ri, const T *&rv, int &nb,
                       int &st) {
        a = T(0); nb = 0; st = 0; ri = B.idx; rv = B.val;
        if (t < na) {
          const int k = A.idx[(size_t)r * A.w + t];
          if ((unsigned)k < (unsigned)B.n) {
            a = alpha_r * A.val[(size_t)r * A.w + t];
            nb = min(B.nnz[k], B.w);
            st = up.tp ? min(max(up.tp[(size_t)r * A.w + t], 0), nb) : 0;
            ri = B.idx + (size_t)k * B.w;
            rv = B.val + (size_t)k * B.w;
          }
        }
#pragma unroll
        for (int u = 0; u < kWinPre; ++u) {
          const int q = st + threadIdx.x + u * kWinThreads;
          jr[u] = q < nb ? __ldg(ri + q) : -1;
          vr[u] = q < nb ? __ldg(rv + q) : T(0);
        }
      };
      fetch(0, cj, cv, ca, crow, cvrow, cnb, cst);
      for (int t = 0; t < na; ++t) {
        fetch(t + 1, nj, nv, an, nrow, nvrow, nnb, nst);
#pragma unroll
        for (int u = 0; u < kWinPre; ++u) {
          const int j = cj[u];
          if (j >= lo && j <= hi) acc[j - lo] = fmadd(ca, cv[u], acc[j - lo]);
        }
        // entries beyond the prefetched ones (source rows longer than kWinPre * threads)
        for (int q = cst + threadIdx.x + kWinPre * kWinThreads; q < cnb; q += kWinThreads) {
          const int j = __ldg(crow + q);
          if (j >= lo && j <= hi) acc[j - lo] = fmadd(ca, __ldg(cvrow + q), acc[j - lo]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kWinPre; ++u) {
          cj[u] = nj[u];
          cv[u] = nv[u];
        }
        ca = an; crow = nrow; cvrow = nvrow; cnb = nnb; cst = nst;
      }
    }
    // scan the window in column order: structural entries that pass the drop rule
    int base = 0;
    double d = 0.0, f = 0.0;
    for (int c0 = 0; c0 < span; c0 += blockDim.x) {
      const int c = c0 + threadIdx.x;
      bool keep = false;
      T v = T(0);
      if (c < span && (!marks || ((touched[c >> 5] >> (c & 31)) & 1u))) {
        v = acc[c];
        keep = marks || mag_bits(v) > tb;
      }
      int total;
      const int pos = base + block_exclusive_scan_ballot<T>(keep, s_warp, total);
      if (keep) {
        const int j = lo + c;
        if (pos < Out.w) {
          Out.idx[(size_t)r * Out.w + pos] = j;
          Out.val[(size_t)r * Out.w + pos] = v;
        }
        const double dv = (double)v;
        if (j == r) d += dv;
        f = fma(dv, dv, f);
      }
      base += total;
    }
    d = warp_sum(d);
    f = warp_sum(f);
    if (lane == 0) { s_d[wid] = d; s_f[wid] = f; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double dd = 0.0, ff = 0.0;
      for (int w = 0; w < nwarp; ++w) { dd += s_d[w]; ff += s_f[w]; }
      lmax = max(lmax, base);
      if (base > Out.w) {
        ++lover;
        rowstat[r] = make_double2(0.0, 0.0);
      } else {
        Out.nnz[r] = base;
        rowstat[r] = make_double2(dd, ff);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (lmax) atomicMax(&ctl->max_count, lmax);
    if (lover) atomicAdd(&ctl->overflow_rows, lover);
  }
}

// ------------------------------------------------------------------ add
// A <- drop_tau(alpha*A + beta*B), warp per row, table of 2^11 slots.
template <typename T>
__global__ void __launch_bounds__(HashCfg<T, 11>::WARPS * 32)
    add_hash_kernel(EllOut<T> A, EllView<T> B, T alpha, T beta, T tau, double2 *__restrict__ rowstat,
                    SpgemmCtl *__restrict__ ctl, int *__restrict__ fb_list) {
  using Cfg = HashCfg<T, 11>;
  constexpr int TS = Cfg::TS;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int *keys = reinterpret_cast<int *>(smem + (size_t)wid * Cfg::BYTES_PER_WARP);
  T *vals = reinterpret_cast<T *>(keys + TS);
  const int nw = gridDim.x * Cfg::WARPS;
  int wmax = 0, wover = 0;
  for (int r = blockIdx.x * Cfg::WARPS + wid; r < A.n; r += nw) {
    const int na = min(A.nnz[r], A.w), nb = min(B.nnz[r], B.w);
    if (na + nb > Cfg::LIMIT) {
      if (lane == 0) {
        const int p = atomicAdd(&ctl->n_fallback, 1);
        fb_list[p] = r;
      }
      continue;
    }
    for (int s = lane * 4; s < TS; s += 128) *reinterpret_cast<int4 *>(keys + s) = make_int4(-1, -1, -1, -1);
    __syncwarp();
    int ins = 0;
    for (int s = lane; s < na; s += 32) {
      const int j = A.idx[(size_t)r * A.w + s];
      if ((unsigned)j >= (unsigned)A.n) continue;
      const int h = find_or_insert<11>(keys, vals, j, ins);
      if (h >= 0) vals[h] = alpha * A.val[(size_t)r * A.w + s];
    }
    __syncwarp();
    for (int s = lane; s < nb; s += 32) {
      const int j = B.idx[(size_t)r * B.w + s];
      if ((unsigned)j >= (unsigned)A.n) continue;
      const int h = find_or_insert<11>(keys, vals, j, ins);
      if (h >= 0) vals[h] = fmadd(beta, B.val[(size_t)r * B.w + s], vals[h]);
    }
    __syncwarp();
    const int nk = compact_table<T, TS>(keys, vals, tau, lane);
    wmax = max(wmax, nk);
    if (nk > A.w) {
      ++wover;
      if (lane == 0) rowstat[r] = make_double2(0.0, 0.0);
      continue;
    }
    sort_prefix<T>(keys, vals, nk, lane);
    double dsum = 0.0, fsum = 0.0;
    for (int s = lane; s < nk; s += 32) {
      const int key = keys[s];
      const T v = vals[s];
      A.idx[(size_t)r * A.w + s] = key;
      A.val[(size_t)r * A.w + s] = v;
      const double dv = (double)v;
      if (key == r) dsum += dv;
      fsum = fma(dv, dv, fsum);
    }
    dsum = warp_sum(dsum);
    fsum = warp_sum(fsum);
    if (lane == 0) {
      A.nnz[r] = nk;
      rowstat[r] = make_double2(dsum, fsum);
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (wmax) atomicMax(&ctl->max_count, wmax);
    if (wover) atomicAdd(&ctl->overflow_rows, wover);
  }
}

template <typename T>
__global__ void __launch_bounds__(kDenseThreads)
    add_dense_kernel(EllOut<T> A, EllView<T> B, T alpha, T beta, T tau, double2 *__restrict__ rowstat,
                     SpgemmCtl *__restrict__ ctl, const int *__restrict__ fb_list, T *__restrict__ acc_all,
                     int *__restrict__ mark_all) {
  __shared__ int s_warp[kDenseThreads / 32];
  __shared__ double s_d[kDenseThreads / 32], s_f[kDenseThreads / 32];
  const int n = A.n;
  const int nfb = *((volatile int *)&ctl->n_fallback);
  T *acc = acc_all + (size_t)blockIdx.x * n;
  int *mark = mark_all + (size_t)blockIdx.x * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int lmax = 0, lover = 0;
  for (int q = blockIdx.x; q < nfb; q += gridDim.x) {
    const int r = fb_list[q];
    const int na = min(A.nnz[r], A.w), nb = min(B.nnz[r], B.w);
    for (int s = threadIdx.x; s < na; s += blockDim.x) {
      const int j = A.idx[(size_t)r * A.w + s];
      if ((unsigned)j >= (unsigned)n) continue;
      mark[j] = 1;
      acc[j] = alpha * A.val[(size_t)r * A.w + s];
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nb; s += blockDim.x) {
      const int j = B.idx[(size_t)r * B.w + s];
      if ((unsigned)j >= (unsigned)n) continue;
      mark[j] = 1;
      acc[j] = fmadd(beta, B.val[(size_t)r * B.w + s], acc[j]);
    }
    __syncthreads();
    int base = 0;
    double d = 0.0, f = 0.0;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
      const int j = c0 + threadIdx.x;
      bool keep = false;
      T v = T(0);
      if (j < n && mark[j] != -1) {
        v = acc[j];
        keep = keep_value(v, tau);
        mark[j] = -1;
        acc[j] = T(0);
      }
      int total;
      const int pos = base + block_exclusive_scan_ballot<T>(keep, s_warp, total);
      if (keep) {
        if (pos < A.w) {
          A.idx[(size_t)r * A.w + pos] = j;
          A.val[(size_t)r * A.w + pos] = v;
        }
        const double dv = (double)v;
        if (j == r) d += dv;
        f += dv * dv;
      }
      base += total;
    }
    d = warp_sum(d);
    f = warp_sum(f);
    if (lane == 0) { s_d[wid] = d; s_f[wid] = f; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double dd = 0.0, ff = 0.0;
      for (int w = 0; w < nwarp; ++w) { dd += s_d[w]; ff += s_f[w]; }
      rowstat[r] = make_double2(dd, ff);
      lmax = max(lmax, base);
      if (base > A.w) ++lover; else A.nnz[r] = base;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (lmax) atomicMax(&ctl->max_count, lmax);
    if (lover) atomicAdd(&ctl->overflow_rows, lover);
  }
}

// ------------------------------------------------------------------ launchers
namespace {

constexpr int kFallbackSlots = 64;

template <typename K>
int set_smem(K kernel, int bytes) {
  SP2_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return SP2_OK;
}

// Launches the hash kernel over all rows (row_list == nullptr) or over a device-side list.
template <typename T, int LOG2T, int QM>
int launch_hash(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, const int *row_list, const int *row_count,
                int *fb, int *fb_count, cudaStream_t s) {
  using Cfg = HashCfg<T, LOG2T>;
  auto kern = spgemm_hash_kernel<T, LOG2T, QM>;
  static DeviceOnce once;
  const int dev = current_device();
  SP2_TRY(device_once(once, dev, [&](int &occ) {
    SP2_TRY(set_smem(kern, Cfg::SMEM));
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Cfg::WARPS * 32, Cfg::SMEM));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  const long long cap = (long long)num_sms() * once.value[dev];
  long long blocks = row_list ? cap : ((long long)a.A->n + Cfg::WARPS - 1) / Cfg::WARPS;
  int grid = (int)(blocks < cap ? blocks : cap);
  if (grid < 1) grid = 1;
  const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
  const int cls = row_list ? SP2_PROF_LARGE : SP2_PROF_SPGEMM;
  prof_begin(cls, s);
  kern<<<grid, Cfg::WARPS * 32, Cfg::SMEM, s>>>(view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha,
                                               (T)a.beta, (T)a.tau, a.Add != nullptr && a.beta != 0.0, a.bv, a.up,
                                               rowstat, ctl, row_list, row_count, fb, fb_count);
  note_launch();
  prof_end(cls, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

template <typename T, int R, int QW, bool KEEPZ, int SZ = 0>
int launch_block(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s,
                 PassRows rows = PassRows{}) {
  using Geo = BlockGeo<T, R, SZ>;
  auto kern = spgemm_block_kernel<T, R, QW, KEEPZ, SZ>;
  static DeviceOnce once;
  const int dev = current_device();
  SP2_TRY(device_once(once, dev, [&](int &occ) {
    SP2_TRY(set_smem(kern, Geo::SMEM));
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Geo::WARPS * 32, Geo::SMEM));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  const long long cap = (long long)num_sms() * once.value[dev];
  // a row list's length is on the device: the whole resident grid, idle CTAs exit at once
  const long long blocks = rows.list ? cap : ((long long)a.A->n + Geo::GROUPS - 1) / Geo::GROUPS;
  int grid = (int)(blocks < cap ? blocks : cap);
  if (grid < 1) grid = 1;
  const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
  const int cls = rows.list ? SP2_PROF_CASCADE : SP2_PROF_SPGEMM;
  prof_begin(cls, s);
  kern<<<grid, Geo::WARPS * 32, Geo::SMEM, s>>>(view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha,
                                               (T)a.beta, (T)a.tau, a.Add != nullptr && a.beta != 0.0, a.bv, a.up,
                                               rowstat, ctl, fb, fb_count, a.route, rows);
  note_launch();
  prof_end(cls, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

template <typename T, int QM, int S, bool KEEPZ, int SZ = 0>
int launch_super(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s,
                 PassRows rows = PassRows{}) {
  using Geo = BlockGeo<T, 1, SZ>;
  auto kern = spgemm_super_kernel<T, QM, S, KEEPZ, SZ>;
  static DeviceOnce once;
  const int dev = current_device();
  SP2_TRY(device_once(once, dev, [&](int &occ) {
    SP2_TRY(set_smem(kern, Geo::SMEM));
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Geo::WARPS * 32, Geo::SMEM));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  const long long cap = (long long)num_sms() * once.value[dev];
  // a row list's length is on the device: the whole resident grid, idle CTAs exit at once
  const long long blocks = rows.list ? cap : ((long long)a.A->n + Geo::GROUPS - 1) / Geo::GROUPS;
  int grid = (int)(blocks < cap ? blocks : cap);
  if (grid < 1) grid = 1;
  const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
  const int cls = rows.list ? SP2_PROF_CASCADE : SP2_PROF_SPGEMM;
  prof_begin(cls, s);
  kern<<<grid, Geo::WARPS * 32, Geo::SMEM, s>>>(view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha,
                                               (T)a.beta, (T)a.tau, a.Add != nullptr && a.beta != 0.0, a.bv, a.up,
                                               rowstat, ctl, fb, fb_count, a.route, rows);
  note_launch();
  prof_end(cls, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

template <typename T>
int launch_super_auto(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s,
                      PassRows rows = PassRows{}) {
  constexpr int QM = sizeof(T) == 8 ? 6 : 6;
  return a.tau == 0.0 ? launch_super<T, QM, 2, true>(a, rowstat, ctl, fb, fb_count, s, rows)
                      : launch_super<T, QM, 2, false>(a, rowstat, ctl, fb, fb_count, s, rows);
}

// Compact variants for the upper-triangle rows of symmetric products: fewer accumulator
// slots per row and fewer warps per row (2 for the column blocks), more rows per SM.
template <typename T, int SZ>
int launch_block_compact(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count,
                         cudaStream_t s, PassRows rows = PassRows{}) {
  return a.tau == 0.0 ? launch_block<T, 2, 2, true, SZ>(a, rowstat, ctl, fb, fb_count, s, rows)
                      : launch_block<T, 2, 2, false, SZ>(a, rowstat, ctl, fb, fb_count, s, rows);
}
template <typename T, int SZ>
int launch_super_compact(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count,
                         cudaStream_t s, PassRows rows = PassRows{}) {
  return a.tau == 0.0 ? launch_super<T, 3, 2, true, SZ>(a, rowstat, ctl, fb, fb_count, s, rows)
                      : launch_super<T, 3, 2, false, SZ>(a, rowstat, ctl, fb, fb_count, s, rows);
}

// Block first pass with R warps per row; the register slots per warp cover the width of B.
template <typename T, int R>
int launch_block_r(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s,
                   PassRows rows = PassRows{}) {
  constexpr int QW = (R == 1) ? 8 : (R == 2 ? 4 : 2);
  return a.tau == 0.0 ? launch_block<T, R, QW, true>(a, rowstat, ctl, fb, fb_count, s, rows)
                      : launch_block<T, R, QW, false>(a, rowstat, ctl, fb, fb_count, s, rows);
}

// First pass over every row (path: 0 automatic, 1/2/4 column blocks with that many
// warps per row, 10..12 hash table of 2^path slots per warp), then the deferred rows in
// a one-warp 2^14-slot hash table.
// Window bin over the rows of a device-side list; rows wider than the window go to out.
template <typename T>
int launch_window(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, const int *in, const int *in_count, int *out,
                  int *out_count, cudaStream_t s) {
  using Cfg = WinCfg<T>;
  static DeviceOnce once;
  SP2_TRY(device_once(once, current_device(), [&](int &) { return set_smem(spgemm_window_kernel<T>, Cfg::SMEM); }));
  const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
  prof_begin(SP2_PROF_LARGE, s);
  spgemm_window_kernel<T><<<num_sms(), kWinThreads, Cfg::SMEM, s>>>(
      view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha, (T)a.beta, (T)a.tau,
      a.Add != nullptr && a.beta != 0.0, a.bv, a.up, rowstat, ctl, in, in_count, out, out_count);
  note_launch();
  prof_end(SP2_PROF_LARGE, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

template <typename T, int QM>
int launch_bins(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb1, int *fbw, int *fb2, int path,
                cudaStream_t s) {
  int rc = SP2_OK;
  switch (path) {
    case 1: rc = launch_block_r<T, 1>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    case 4: rc = launch_block_r<T, 4>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    case 10: rc = launch_hash<T, 10, QM>(a, rowstat, ctl, nullptr, nullptr, fb1, &ctl->n_fallback, s); break;
    case 11: rc = launch_hash<T, 11, QM>(a, rowstat, ctl, nullptr, nullptr, fb1, &ctl->n_fallback, s); break;
    case 12: rc = launch_hash<T, 12, QM>(a, rowstat, ctl, nullptr, nullptr, fb1, &ctl->n_fallback, s); break;
    case 2: rc = launch_block_r<T, 2>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    case 3: rc = launch_super_auto<T>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    case 7: rc = launch_block_compact<T, 1>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    case 8: rc = launch_super_compact<T, 1>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    case 9: rc = launch_tile<T>(a, rowstat, ctl, fb1, &ctl->n_fallback, s); break;
    default: {  // automatic: the variant measured fastest on the 3D tight-binding products
                // (FP64: column blocks, 4 warps per row, 2 in the compact form; FP32: one warp
                // per row, two k steps per pass)
      // The upper triangle of a symmetric product runs a cascade from compact_level on:
      // the tight compact pass over every row, the loose one over the rows that outgrew
      // it, the full-row pass over the rows that outgrew that; each pass is a first pass
      // over a device-side list (fb1 and fbw alternate), so a long row costs one pass of
      // its level instead of a CTA of the window bin.  Full rows: the full-row pass alone.
      const int first = cascade_start(a.A->n, a.up.tp != nullptr, a.compact_level);
      int *bufs[2] = {fb1, fbw};
      int cur = 0;
      PassRows rows{};
      for (int lv = first; lv <= 2 && rc == SP2_OK; ++lv) {
        rows.level = lv;
        int *out = bufs[cur];
        int *out_count = lv == 0 ? &ctl->n_level1 : (lv == 1 ? &ctl->n_level2 : &ctl->n_fallback);
        if (lv == 0)
          rc = sizeof(T) == 8 ? launch_block_compact<T, 1>(a, rowstat, ctl, out, out_count, s, rows)
                              : launch_super_compact<T, 1>(a, rowstat, ctl, out, out_count, s, rows);
        else if (lv == 1)
          rc = sizeof(T) == 8 ? launch_block_compact<T, 2>(a, rowstat, ctl, out, out_count, s, rows)
                              : launch_super_compact<T, 2>(a, rowstat, ctl, out, out_count, s, rows);
        else
          rc = sizeof(T) == 8 ? launch_block_r<T, 4>(a, rowstat, ctl, out, out_count, s, rows)
                              : launch_super_auto<T>(a, rowstat, ctl, out, out_count, s, rows);
        rows.list = out;
        rows.count = out_count;
        cur ^= 1;
      }
      // the rows the full-row pass passed on: bins as below, from the list it wrote
      if (rc == SP2_OK)
        rc = launch_window<T>(a, rowstat, ctl, rows.list, &ctl->n_fallback, bufs[cur], &ctl->n_fallbackw, s);
      if (rc == SP2_OK)
        rc = launch_hash<T, 14, QM>(a, rowstat, ctl, bufs[cur], &ctl->n_fallbackw, fb2, &ctl->n_fallback2, s);
      return rc;
    }
  }
  // deferred rows: a dense window per CTA when the row's span fits it, then the 2^14-slot
  // table, then dense global rows
  if (rc == SP2_OK) rc = launch_window<T>(a, rowstat, ctl, fb1, &ctl->n_fallback, fbw, &ctl->n_fallbackw, s);
  if (rc == SP2_OK)
    rc = launch_hash<T, 14, QM>(a, rowstat, ctl, fbw, &ctl->n_fallbackw, fb2, &ctl->n_fallback2, s);
  return rc;
}

template <typename T>
int multiply_t(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, cudaStream_t s);

// Symmetric product: upper rows into a scratch matrix U, then mirrored into a.Out.  U is
// as wide as the output; if an upper row does not fit (so the output cannot fit either),
// the first pass is repeated with U as wide as the longest upper row, so that the
// reported required width stays exact -- except while a stream is being captured (the
// batched loop regrows on its own), where the report is then a lower bound.
template <typename T>
int multiply_sym_t(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, cudaStream_t s) {
  const int n = a.A->n;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SP2_CUDA(cudaStreamIsCapturing(s, &cap));
  int uw = a.Out->width;
  for (int attempt = 0;; ++attempt) {
    const size_t bytes = sym_scratch_bytes(n, a.A->width, uw, a.A->dtype);
    unsigned char *scr = static_cast<unsigned char *>(a.sym_prealloc);
    const bool own = !scr || a.sym_prealloc_bytes < bytes;
    if (own && cap != cudaStreamCaptureStatusNone) return fail(SP2E_ARG, "multiply: symmetric scratch too small");
    if (own) SP2_TRY(dev_alloc((void **)&scr, bytes, s));
    // layout: U.val, U.idx, U.nnz, tp, tpd, work (each 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t b) { unsigned char *q = scr + off; off += round_up_sz(b, 256); return q; };
    ellpack_t U{};
    U.n = n;
    U.width = uw;
    U.dtype = a.A->dtype;
    U.owner = 0;
    U.val = take(sizeof(T) * (size_t)n * uw);
    U.idx = reinterpret_cast<int *>(take(sizeof(int) * (size_t)n * uw));
    U.nnz = reinterpret_cast<int *>(take(sizeof(int) * (size_t)n));
    int *tp = reinterpret_cast<int *>(take(sizeof(int) * (size_t)n * a.A->width));
    int *tpd = reinterpret_cast<int *>(take(sizeof(int) * (size_t)n));
    int *work = reinterpret_cast<int *>(take(sizeof(int) * (3 * (size_t)n + 1)));
    int rc = SP2_OK;
    cudaError_t e = cudaMemsetAsync(U.nnz, 0, sizeof(int) * (size_t)n, s);
    if (e == cudaSuccess && attempt > 0) e = cudaMemsetAsync(ctl, 0, sizeof(SpgemmCtl), s);
    if (e != cudaSuccess) rc = cuda_fail(e, "multiply (symmetric)", __FILE__, __LINE__);
    if (rc == SP2_OK) rc = upper_start_async(a.A, tp, tpd, s);
    if (rc == SP2_OK) {
      MultiplyArgs a1 = a;
      a1.sym = false;
      a1.Out = &U;
      a1.up = Upper{tp, tpd};
      rc = multiply_t<T>(a1, rowstat, ctl, s);
    }
    SpgemmCtl h{};
    if (rc == SP2_OK && cap == cudaStreamCaptureStatusNone && attempt == 0) {
      e = cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = cuda_fail(e, "multiply (symmetric)", __FILE__, __LINE__);
    }
    if (rc == SP2_OK && h.overflow_rows > 0 && h.max_count > uw) {  // an upper row did not fit: widen U, redo
      if (own) dev_free(scr, s);
      uw = round_up(h.max_count, 32);
      continue;
    }
    if (rc == SP2_OK) rc = mirror_async(&U, a.Out, a.bv, work, rowstat, ctl, s);
    if (own) dev_free(scr, s);
    return rc;
  }
}

template <typename T>
int multiply_t(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, cudaStream_t s) {
  if (a.sym) return multiply_sym_t<T>(a, rowstat, ctl, s);
  const int n = a.A->n;
  int *fb = a.fb_prealloc;
  if (!fb) SP2_TRY(dev_alloc((void **)&fb, 3 * sizeof(int) * (size_t)n, s));
  int *fb1 = fb, *fbw = fb + n, *fb2 = fb + 2 * (size_t)n;
  const int qm_need = (a.B->width + 31) / 32;
  int rc = qm_need <= 4 ? launch_bins<T, 4>(a, rowstat, ctl, fb1, fbw, fb2, a.path, s)
                        : launch_bins<T, 8>(a, rowstat, ctl, fb1, fbw, fb2, a.path, s);
  if (rc == SP2_OK) {
    // bin 2: rows beyond the largest table, dense global-memory rows
    void *acc = nullptr;
    int *mark = nullptr;
    int slots = kFallbackSlots;
    if (slots > n) slots = n;
    rc = fallback_scratch(a.Out->n, a.A->dtype, slots, &acc, &mark, s);  // one dense row per slot
    if (rc == SP2_OK) {
      const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
      spgemm_dense_kernel<T><<<slots, kDenseThreads, 0, s>>>(
          view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha, (T)a.beta, (T)a.tau,
          a.Add != nullptr && a.beta != 0.0, a.bv, a.up, rowstat, ctl, fb2, &ctl->n_fallback2, (T *)acc, mark);
      note_launch();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "spgemm_dense_kernel", __FILE__, __LINE__);
    }
  }
  if (!a.fb_prealloc) dev_free(fb, s);
  return rc;
}

template <typename T>
int add_t(ellpack_t *A, const ellpack_t *B, double alpha, double beta, double tau, double2 *rowstat,
          SpgemmCtl *ctl, cudaStream_t s) {
  using Cfg = HashCfg<T, 11>;
  const int n = A->n;
  int *fb = nullptr;
  SP2_TRY(dev_alloc((void **)&fb, sizeof(int) * (size_t)n, s));
  int rc = set_smem(add_hash_kernel<T>, Cfg::SMEM);
  if (rc == SP2_OK) {
    long long blocks = ((long long)n + Cfg::WARPS - 1) / Cfg::WARPS;
    long long cap = (long long)num_sms() * 2;
    int grid = (int)(blocks < cap ? blocks : cap);
    add_hash_kernel<T><<<grid, Cfg::WARPS * 32, Cfg::SMEM, s>>>(outview<T>(A), view<T>(B), (T)alpha, (T)beta,
                                                               (T)tau, rowstat, ctl, fb);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "add_hash_kernel", __FILE__, __LINE__);
  }
  if (rc == SP2_OK) {
    void *acc = nullptr;
    int *mark = nullptr;
    int slots = kFallbackSlots < n ? kFallbackSlots : n;
    rc = fallback_scratch(n, A->dtype, slots, &acc, &mark, s);
    if (rc == SP2_OK) {
      add_dense_kernel<T><<<slots, kDenseThreads, 0, s>>>(outview<T>(A), view<T>(B), (T)alpha, (T)beta, (T)tau,
                                                          rowstat, ctl, fb, (T *)acc, mark);
      note_launch();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "add_dense_kernel", __FILE__, __LINE__);
    }
  }
  dev_free(fb, s);
  return rc;
}

}  // namespace

int multiply_async(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, cudaStream_t s) {
  SP2_CUDA(cudaMemsetAsync(ctl, 0, sizeof(SpgemmCtl), s));
  if (a.A->dtype == SP2_F64) return multiply_t<double>(a, rowstat, ctl, s);
  return multiply_t<float>(a, rowstat, ctl, s);
}

int add_async(ellpack_t *A, const ellpack_t *B, double alpha, double beta, double tau, double2 *rowstat,
              SpgemmCtl *ctl, cudaStream_t s) {
  SP2_CUDA(cudaMemsetAsync(ctl, 0, sizeof(SpgemmCtl), s));
  if (A->dtype == SP2_F64) return add_t<double>(A, B, alpha, beta, tau, rowstat, ctl, s);
  return add_t<float>(A, B, alpha, beta, tau, rowstat, ctl, s);
}

}  // namespace sp2

// ==================================================================== C ABI
using namespace sp2;

namespace {
bool same_arrays(const ellpack_t *x, const ellpack_t *y) {
  return x->idx == y->idx || x->val == y->val || x->nnz == y->nnz;
}

int check_tau(double tau, const char *who) {
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(SP2E_ARG, "%s: tau must be finite and >= 0", who);
  return SP2_OK;
}

int finish_step(SpgemmCtl *ctl, double2 *rowstat, const ellpack_t *out, cudaStream_t s, int32_t *required_width,
                const char *who) {
  StepResult *dres = nullptr;
  SP2_TRY(dev_alloc((void **)&dres, sizeof(StepResult), s));
  launch_reduce_rows(rowstat, out->nnz, out->n, ctl, dres, s);
  StepResult h;
  cudaError_t e = cudaMemcpyAsync(&h, dres, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(dres, s);
  if (e != cudaSuccess) return cuda_fail(e, who, __FILE__, __LINE__);
  if (required_width) *required_width = h.max_count;
  if (h.overflow_rows > 0)
    return fail(SP2E_OVERFLOW, "%s: %d row(s) need %d slots, output width is %d", who, h.overflow_rows, h.max_count,
                out->width);
  return SP2_OK;
}
}  // namespace

extern "C" int ellpack_multiply(const ellpack_t *A, const ellpack_t *B, ellpack_t *C, double alpha, double beta,
                                double tau, void *stream, int32_t *required_width) {
  SP2_TRY(check_matrix(A, "ellpack_multiply: A"));
  SP2_TRY(check_matrix(B, "ellpack_multiply: B"));
  SP2_TRY(check_matrix(C, "ellpack_multiply: C"));
  SP2_TRY(check_tau(tau, "ellpack_multiply"));
  if (A->n != B->n || A->n != C->n) return fail(SP2E_ARG, "ellpack_multiply: sizes differ (%d, %d, %d)", A->n, B->n, C->n);
  if (A->dtype != B->dtype || A->dtype != C->dtype) return fail(SP2E_ARG, "ellpack_multiply: dtypes differ");
  if (same_arrays(C, A) || same_arrays(C, B)) return fail(SP2E_ARG, "ellpack_multiply: C aliases A or B");
  if (!isfinite(alpha) || !isfinite(beta)) return fail(SP2E_ARG, "ellpack_multiply: alpha/beta not finite");
  cudaStream_t s = as_stream(stream);
  double2 *rowstat = nullptr;
  SpgemmCtl *ctl = nullptr;
  SP2_TRY(dev_alloc((void **)&rowstat, sizeof(double2) * (size_t)A->n, s));
  int rc = dev_alloc((void **)&ctl, sizeof(SpgemmCtl), s);
  if (rc == SP2_OK) {
    MultiplyArgs a{A, B, beta != 0.0 ? C : nullptr, C, alpha, beta, tau, 0};
    rc = multiply_async(a, rowstat, ctl, s);
    if (rc == SP2_OK) rc = finish_step(ctl, rowstat, C, s, required_width, "ellpack_multiply");
  }
  dev_free(rowstat, s);
  dev_free(ctl, s);
  return rc;
}

extern "C" int ellpack_multiply_block(const ellpack_t *A, int32_t row0, const ellpack_t *B, const ellpack_t *C,
                                      ellpack_t *Out, double alpha, double beta, double tau, int32_t *required_width,
                                      double *trace, double *frobenius2, void *stream) {
  SP2_TRY(check_matrix(A, "ellpack_multiply_block: A"));
  SP2_TRY(check_matrix(B, "ellpack_multiply_block: B"));
  SP2_TRY(check_matrix(Out, "ellpack_multiply_block: Out"));
  if (beta != 0.0) SP2_TRY(check_matrix(C, "ellpack_multiply_block: C"));
  SP2_TRY(check_tau(tau, "ellpack_multiply_block"));
  if (A->n != Out->n || (beta != 0.0 && C->n != A->n))
    return fail(SP2E_ARG, "ellpack_multiply_block: A, C and Out must hold the same rows");
  if (row0 < 0 || (long long)row0 + A->n > (long long)B->n)
    return fail(SP2E_ARG, "ellpack_multiply_block: rows %d .. %lld are not rows of B (n = %d)", row0,
                (long long)row0 + A->n - 1, B->n);
  if (A->dtype != B->dtype || A->dtype != Out->dtype || (beta != 0.0 && C->dtype != A->dtype))
    return fail(SP2E_ARG, "ellpack_multiply_block: dtypes differ");
  if (same_arrays(Out, A) || same_arrays(Out, B) || (beta != 0.0 && same_arrays(Out, C)))
    return fail(SP2E_ARG, "ellpack_multiply_block: Out aliases an input");
  if (!isfinite(alpha) || !isfinite(beta)) return fail(SP2E_ARG, "ellpack_multiply_block: alpha/beta not finite");
  cudaStream_t s = as_stream(stream);
  const int nb = A->n;
  double2 *rowstat = nullptr;
  SpgemmCtl *ctl = nullptr;
  StepResult *dres = nullptr;
  SP2_TRY(dev_alloc((void **)&rowstat, sizeof(double2) * (size_t)nb, s));
  int rc = dev_alloc((void **)&ctl, sizeof(SpgemmCtl), s);
  if (rc == SP2_OK) rc = dev_alloc((void **)&dres, sizeof(StepResult), s);
  if (rc == SP2_OK) {
    // the product's columns are B's rows: the output view spans B->n columns, while the
    // kernels write only A's rows
    ellpack_t wide = *Out;
    wide.n = B->n;
    MultiplyArgs a{A, B, beta != 0.0 ? C : nullptr, &wide, alpha, beta, tau, 0};
    rc = multiply_async(a, rowstat, ctl, s);
    // statistics of the block's rows: the diagonal of local row r is column row0 + r
    if (rc == SP2_OK) rc = rowstat_async(Out, rowstat, s, row0);
    if (rc == SP2_OK) {
      launch_reduce_rows(rowstat, Out->nnz, nb, ctl, dres, s);
      StepResult h;
      cudaError_t e = cudaMemcpyAsync(&h, dres, sizeof(h), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "ellpack_multiply_block", __FILE__, __LINE__);
      } else {
        if (required_width) *required_width = h.max_count;
        if (trace) *trace = h.tr;
        if (frobenius2) *frobenius2 = h.fro;
        if (h.overflow_rows > 0)
          rc = fail(SP2E_OVERFLOW, "ellpack_multiply_block: %d row(s) need %d slots, output width is %d",
                    h.overflow_rows, h.max_count, Out->width);
      }
    }
  }
  dev_free(rowstat, s);
  dev_free(ctl, s);
  dev_free(dres, s);
  return rc;
}

extern "C" int ellpack_add(ellpack_t *A, const ellpack_t *B, double alpha, double beta, double tau, void *stream,
                           int32_t *required_width) {
  SP2_TRY(check_matrix(A, "ellpack_add: A"));
  SP2_TRY(check_matrix(B, "ellpack_add: B"));
  SP2_TRY(check_tau(tau, "ellpack_add"));
  if (A->n != B->n) return fail(SP2E_ARG, "ellpack_add: sizes differ");
  if (A->dtype != B->dtype) return fail(SP2E_ARG, "ellpack_add: dtypes differ");
  if (same_arrays(A, B)) return fail(SP2E_ARG, "ellpack_add: A and B alias");
  if (!isfinite(alpha) || !isfinite(beta)) return fail(SP2E_ARG, "ellpack_add: alpha/beta not finite");
  cudaStream_t s = as_stream(stream);
  double2 *rowstat = nullptr;
  SpgemmCtl *ctl = nullptr;
  SP2_TRY(dev_alloc((void **)&rowstat, sizeof(double2) * (size_t)A->n, s));
  int rc = dev_alloc((void **)&ctl, sizeof(SpgemmCtl), s);
  if (rc == SP2_OK) {
    rc = add_async(A, B, alpha, beta, tau, rowstat, ctl, s);
    if (rc == SP2_OK) rc = finish_step(ctl, rowstat, A, s, required_width, "ellpack_add");
  }
  dev_free(rowstat, s);
  dev_free(ctl, s);
  return rc;
}
