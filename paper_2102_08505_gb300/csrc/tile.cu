// tile.cu -- SpGEMM first pass over tiles of consecutive rows that share one column index.
//
// C_i = drop_tau(alpha * sum_k A_ik B_k + beta * Add_i): the "ELLPACK X2" product of
// Section "Performance Evaluation using System Matrices", with the "SP2 Loop Misc" update
// fused (Section "Performance Evaluation using an ExaSP2 Application").
//
// Design (GB300).  Consecutive rows of a locality-ordered matrix reach mostly the same
// source rows and the same output columns.  A CTA takes TT such rows and builds, once for
// all of them, U = the sorted set of output columns they can reach: the columns of every
// source row k that one of them uses (read from the tile's first position in the upper-
// triangle mode of symmetric products) and of their addend rows.  U is held as a table of
// 32-column groups: group g = j >> 5 -> (bit mask of its members, rank in U of its first
// member), so the position of column j in U is rank + popc(mask below j).  Each row then
// owns a dense accumulator over U, and one warp computes one row: per entry of a source
// row one read-only table lookup and a plain read-modify-write, no atomics, no barrier
// between source rows (the warp is the only writer of its row).  The epilogue walks the
// groups in column order, so output rows come out sorted without a sort.
//
// Each entry sums its terms in a fixed order (the addend, then the source rows in A's
// order), so results are bitwise reproducible and C_ij = C_ji for a symmetric product.
// A tile whose U does not fit is split in halves; a single row that does not fit goes to
// the deferred-row bins of spgemm.cu.
#include <limits.h>

#include <type_traits>

#include "spgemm_internal.cuh"

namespace sp2 {
namespace {

constexpr unsigned kNoGroup = 0xFFFFFFFFu;

template <typename T>
struct TileCfg {
  static constexpr int TT = 8;                 // rows per full tile = warps per CTA
  static constexpr int CU = 1408;              // accumulator slots per row of a full tile
  static constexpr int SLOTS = TT * CU;        // accumulator slots per CTA
  static constexpr int LOG2GT = 9, GT = 1 << LOG2GT;  // group table entries
  static constexpr int MAXG = 256;             // groups of one sub-tile (sorted by one warp)
  static constexpr int LOG2KT = 10, KT = 1 << LOG2KT;  // source-row table entries
  static constexpr int MAXK = KT - KT / 4;     // source rows of one sub-tile
  static constexpr int QW = 4;                 // register slots of 32 entries per source row
  static constexpr int ACC_BYTES = SLOTS * (int)sizeof(T);
  static constexpr int GENT_BYTES = GT * 16;
  static constexpr int KTAB_BYTES = KT * 8;
  static constexpr int ORDER_BYTES = MAXG * 4;
  static constexpr int SORT_BYTES = MAXG * 8;
  static constexpr int SMEM = ACC_BYTES + GENT_BYTES + KTAB_BYTES + ORDER_BYTES + SORT_BYTES;
  static_assert(ACC_BYTES % 16 == 0, "group table alignment");
};

__device__ __forceinline__ int khash(int k, int log2t) { return (int)(((unsigned)k * 0x9E3779B1u) >> (32 - log2t)); }
__device__ __forceinline__ int gslot0(unsigned g, int log2t) { return (int)((g * 0x85EBCA6Bu) >> (32 - log2t)); }

// Shared-memory tables and arguments of one CTA.
template <typename T, bool KEEPZ>
struct TileCta {
  using Cfg = TileCfg<T>;
  static constexpr int TT = Cfg::TT, GT = Cfg::GT, KT = Cfg::KT, QW = Cfg::QW;
  EllView<T> A, B, Add;
  EllOut<T> Out;
  T alpha, beta, tau;
  int use_add;
  BatchView bv;
  Upper up;
  double2 *rowstat;
  T *acc;            // SLOTS accumulators, clean between sub-tiles
  uint4 *gent;       // group table: {group, member bits, rank of the first member, unused}
  int *kkey, *kst;   // source-row table: k (or -1) and the first position of B_k read
  int *gorder;       // group-table slots in column order
  unsigned long long *sortbuf;
  int *s_flag, *s_nk, *s_ng, *s_nu;
  int lane, w, ncol;
  unsigned lt;
  int wmax, wover;

  __device__ __forceinline__ T clean() const { return KEEPZ ? untouched<T>() : T(0); }

  // Group of column j in the group table, inserted if new; the lanes of a warp that hold
  // columns of one group OR their member bits and one of them updates the entry.
  __device__ __forceinline__ void insert_col(bool on, int j) {
    const unsigned act = __ballot_sync(kFull, on);
    if (on) {
      const unsigned g = (unsigned)j >> 5;
      const unsigned peers = __match_any_sync(act, g);
      const unsigned bits = __reduce_or_sync(peers, 1u << (j & 31));
      if (lane == __ffs(peers) - 1) {
        int h = gslot0(g, Cfg::LOG2GT), slot = -1;
#pragma unroll 1
        for (int p = 0; p < GT; ++p) {
          const unsigned cur = *((volatile unsigned *)&gent[h].x);
          if (cur == g) { slot = h; break; }
          if (cur == kNoGroup) {
            const unsigned old = atomicCAS(&gent[h].x, kNoGroup, g);
            if (old == kNoGroup) { atomicAdd(s_ng, 1); slot = h; break; }
            if (old == g) { slot = h; break; }
          }
          h = (h + 1) & (GT - 1);
        }
        if (slot >= 0) atomicOr(&gent[slot].y, bits);
        else *s_flag = 1;
      }
    }
  }

  // Position of column j in U (j was inserted by the build; -1 if absent, which the build
  // rules out).
  __device__ __forceinline__ int lookup(int j) const {
    const unsigned g = (unsigned)j >> 5;
    int h = gslot0(g, Cfg::LOG2GT);
    uint4 e = gent[h];
#pragma unroll 1
    for (int p = 0; e.x != g && p < GT; ++p) {
      h = (h + 1) & (GT - 1);
      e = gent[h];
    }
    return e.x == g ? (int)e.z + __popc(e.y & ((1u << (j & 31)) - 1u)) : -1;
  }

  // Warp 0: sorts the cnt used groups (keys group << 32 | slot in sortbuf) by column and
  // gives each the rank of its first member in U; the total is |U|.
  template <int E>
  __device__ __forceinline__ void rank_groups(int cnt) {
    unsigned long long key[E];
#pragma unroll
    for (int t = 0; t < E; ++t) key[t] = lane * E + t < cnt ? sortbuf[lane * E + t] : ~0ull;
    warp_bitonic<unsigned long long, E>(key, lane);
    int pc[E], local = 0;
#pragma unroll
    for (int t = 0; t < E; ++t) {
      pc[t] = lane * E + t < cnt ? __popc(gent[(int)(key[t] & 0xFFFFFFFFu)].y) : 0;
      local += pc[t];
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    int run = incl - local;
#pragma unroll
    for (int t = 0; t < E; ++t)
      if (lane * E + t < cnt) {
        const int slot = (int)(key[t] & 0xFFFFFFFFu);
        gent[slot].z = (unsigned)run;
        gorder[lane * E + t] = slot;
        run += pc[t];
      }
    if (lane == 31) *s_nu = incl;
  }

  // One source row from registers: lookups, then the read-modify-writes (the columns of a
  // source row are distinct, so the lanes never collide).  NU occupied register slots.
  template <int NU>
  __device__ __forceinline__ void step_nu(T *racc, const int (&jr)[QW], const T (&vr)[QW], T a) const {
    // first probes of all slots together; a slot whose first probe misses walks on
    int sl[NU];
    uint4 e[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const unsigned g = (unsigned)jr[u] >> 5;
      e[u] = (unsigned)jr[u] < (unsigned)ncol ? gent[gslot0(g, Cfg::LOG2GT)] : make_uint4(g, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const unsigned g = (unsigned)jr[u] >> 5;
      if (e[u].x != g) {
        int h = gslot0(g, Cfg::LOG2GT);
#pragma unroll 1
        for (int p = 0; e[u].x != g && p < GT; ++p) {
          h = (h + 1) & (GT - 1);
          e[u] = gent[h];
        }
      }
      sl[u] = ((unsigned)jr[u] < (unsigned)ncol && e[u].x == g)
                  ? (int)e[u].z + __popc(e[u].y & ((1u << (jr[u] & 31)) - 1u))
                  : -1;
    }
    T old[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) old[u] = sl[u] >= 0 ? racc[sl[u]] : T(0);
#pragma unroll
    for (int u = 0; u < NU; ++u)
      if (sl[u] >= 0) {
        const T o = (KEEPZ && is_untouched(old[u])) ? T(0) : old[u];
        racc[sl[u]] = fmadd(a, vr[u], o);
      }
  }

  __device__ __forceinline__ void step(T *racc, const int (&jr)[QW], const T (&vr)[QW], int nb, T a,
                                       size_t off) const {
    const int nuse = min((nb + 31) >> 5, QW);
    switch (nuse) {
      case 0: break;
      case 1: step_nu<1>(racc, jr, vr, a); break;
      case 2: step_nu<2>(racc, jr, vr, a); break;
      case 3: step_nu<3>(racc, jr, vr, a); break;
      default: step_nu<QW>(racc, jr, vr, a); break;
    }
    for (int q0 = 32 * QW; q0 < nb; q0 += 32) {  // source rows longer than the registers
      const int q = q0 + lane;
      int jt[QW];
      T vt[QW];
      jt[0] = q < nb ? __ldg(B.idx + off + q) : -1;
      vt[0] = q < nb ? __ldg(B.val + off + q) : T(0);
      step_nu<1>(racc, jt, vt, a);
    }
    __syncwarp();  // this source row's updates before the next one's reads
  }

  // Rows [rb, rb + nr) as one sub-tile; false (nothing written) if U does not fit.
  __device__ bool process(int rb, int nr) {
    for (int e = threadIdx.x; e < GT; e += blockDim.x) gent[e] = make_uint4(kNoGroup, 0u, 0u, 0u);
    for (int e = threadIdx.x; e < KT; e += blockDim.x) { kkey[e] = -1; kst[e] = INT_MAX; }
    if (threadIdx.x == 0) { *s_flag = 0; *s_nk = 0; *s_ng = 0; *s_nu = 0; }
    __syncthreads();

    // this warp's row (warp-uniform)
    const int r = rb + w;
    bool active = w < nr;
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (active && bv.row_mat) {
      const int m = bv.row_mat[r];
      active = bv.active[m] != 0;
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    const int na = active ? min(A.nnz[r], A.w) : 0;

    // 1. source rows of the sub-tile, each with the first position any row reads
    for (int s0 = 0; s0 < na; s0 += 32) {
      const int s = s0 + lane;
      if (s < na) {
        const int k = __ldg(A.idx + (size_t)r * A.w + s);
        if ((unsigned)k < (unsigned)B.n) {
          int st = 0;
          if (up.tp) st = min(max(__ldg(up.tp + (size_t)r * A.w + s), 0), min(__ldg(B.nnz + k), B.w));
          int h = khash(k, Cfg::LOG2KT), slot = -1;
#pragma unroll 1
          for (int p = 0; p < KT; ++p) {
            const int cur = *((volatile int *)&kkey[h]);
            if (cur == k) { slot = h; break; }
            if (cur == -1) {
              const int old = atomicCAS(&kkey[h], -1, k);
              if (old == -1) { atomicAdd(s_nk, 1); slot = h; break; }
              if (old == k) { slot = h; break; }
            }
            h = (h + 1) & (KT - 1);
          }
          if (slot >= 0) atomicMin(&kst[slot], st);
          else *s_flag = 1;
        }
      }
    }
    __syncthreads();
    if (*s_flag || *s_nk > Cfg::MAXK) return false;

    // 2. U: the columns of those source rows from their first read position, and of the
    //    addend rows
    for (int e = w; e < KT; e += TT) {
      const int k = kkey[e];
      if (k < 0) continue;
      const int nb = min(__ldg(B.nnz + k), B.w);
      const int *bi = B.idx + (size_t)k * B.w;
      for (int q0 = kst[e]; q0 < nb; q0 += 32) {
        const int q = q0 + lane;
        const int j = q < nb ? __ldg(bi + q) : -1;
        insert_col((unsigned)j < (unsigned)ncol, j);
      }
    }
    int nc = 0, d0 = 0;
    if (active && add_r) {
      nc = min(Add.nnz[r], Add.w);
      d0 = up.tpd ? min(max(up.tpd[r], 0), nc) : 0;
      for (int q0 = d0; q0 < nc; q0 += 32) {
        const int q = q0 + lane;
        const int j = q < nc ? Add.idx[(size_t)r * Add.w + q] : -1;
        insert_col((unsigned)j < (unsigned)ncol, j);
      }
    }
    __syncthreads();
    if (*s_flag || *s_ng > Cfg::MAXG) return false;

    // 3. one warp sorts the groups by column and gives each its rank in U
    if (w == 0) {
      int cnt = 0;
      for (int c = 0; c < GT; c += 32) {
        const unsigned gk = gent[c + lane].x;
        const bool used = gk != kNoGroup;
        const unsigned m = __ballot_sync(kFull, used);
        if (used) sortbuf[cnt + __popc(m & lt)] = ((unsigned long long)gk << 32) | (unsigned)(c + lane);
        cnt += __popc(m);
      }
      __syncwarp();
      if (cnt <= 32) rank_groups<1>(cnt);
      else if (cnt <= 64) rank_groups<2>(cnt);
      else if (cnt <= 128) rank_groups<4>(cnt);
      else rank_groups<8>(cnt);
    }
    __syncthreads();
    const int nu = *s_nu, ng = *s_ng;
    const int cs = Cfg::SLOTS / nr;  // accumulator slots of each row of this sub-tile
    if (nu > cs) return false;
    if (!active) return true;

    // 4. the row: addend, then the source rows in A's order
    T *racc = acc + (size_t)w * cs;
    if (add_r) {
      for (int q0 = d0; q0 < nc; q0 += 32) {
        const int q = q0 + lane;
        if (q < nc) {
          const int j = Add.idx[(size_t)r * Add.w + q];
          const int u = (unsigned)j < (unsigned)ncol ? lookup(j) : -1;
          if (u >= 0) {
            T o = racc[u];
            if (KEEPZ && is_untouched(o)) o = T(0);
            racc[u] = fmadd(beta_r, Add.val[(size_t)r * Add.w + q], o);
          }
        }
      }
      __syncwarp();
    }
    const int *arow_i = A.idx + (size_t)r * A.w;
    const T *arow_v = A.val + (size_t)r * A.w;
    // entries of A's row 32 at a time (current and next chunk): source row, coefficient,
    // first position read and the number of entries read from there
    int ck = 0, cnb = 0, nk_ = 0, nnb = 0, cst = 0, nst = 0;
    T ca = T(0), na_ = T(0);
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
    auto fetch_step = [&](int t, int (&jr)[QW], T (&vr)[QW], int &nb, T &a, size_t &off) {
      int k, st;
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
      off = (size_t)k * B.w + st;
#pragma unroll
      for (int u = 0; u < QW; ++u) {
        const int q = 32 * u + lane;
        jr[u] = q < nb ? __ldg(B.idx + off + q) : -1;
        vr[u] = q < nb ? __ldg(B.val + off + q) : T(0);
      }
    };
    int j0[QW], j1[QW], j2[QW];
    T v0[QW], v1[QW], v2[QW];
    int nb0 = 0, nb1 = 0, nb2 = 0;
    size_t k0 = 0, k1 = 0, k2 = 0;
    T a0 = T(0), a1 = T(0), a2 = T(0);
    if (na > 0) fetch_step(0, j0, v0, nb0, a0, k0);
    if (na > 1) fetch_step(1, j1, v1, nb1, a1, k1);
    for (int t = 0; t < na; t += 3) {
      if (t >= cbase + 32) {  // the next chunk of A's entries becomes current
        ck = nk_; cnb = nnb; ca = na_; cst = nst;
        cbase += 32;
        load_chunk(cbase + 32, nk_, nnb, na_, nst);
      }
      if (t + 2 < na) fetch_step(t + 2, j2, v2, nb2, a2, k2);
      step(racc, j0, v0, nb0, a0, k0);
      if (t + 1 >= na) break;
      if (t + 3 < na) fetch_step(t + 3, j0, v0, nb0, a0, k0);
      step(racc, j1, v1, nb1, a1, k1);
      if (t + 2 >= na) break;
      if (t + 4 < na) fetch_step(t + 4, j1, v1, nb1, a1, k1);
      step(racc, j2, v2, nb2, a2, k2);
    }

    // 5. epilogue: the groups in column order, lane = column within the group; kept
    //    entries are written in order and every slot is left clean for the next tile
    const auto tb = mag_bits(tau);
    const T cl = clean();
    int nk = 0;
    double dsum = 0.0, fsum = 0.0;
    int *oi = Out.idx + (size_t)r * Out.w;
    T *ov = Out.val + (size_t)r * Out.w;
    for (int p = 0; p < ng; ++p) {
      const uint4 e = gent[gorder[p]];
      const int j0c = (int)(e.x << 5);
      if (up.tp && j0c + 31 < r) continue;  // below the diagonal: never touched
      const int j = j0c + lane;
      const bool present = (e.y >> lane) & 1u;
      bool keep = false;
      T v = T(0);
      if (present) {
        const int u = (int)e.z + __popc(e.y & lt);
        v = racc[u];
        keep = KEEPZ ? !is_untouched(v) : mag_bits(v) > tb;
        racc[u] = cl;
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
    return true;
  }
};

template <typename T, bool KEEPZ>
__global__ void __launch_bounds__(TileCfg<T>::TT * 32, 2)
    spgemm_tile_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                       int use_add, BatchView bv, Upper up, int first_rows, const int *__restrict__ tile_list,
                       const int *__restrict__ tile_count, double2 *__restrict__ rowstat,
                       SpgemmCtl *__restrict__ ctl, int *__restrict__ fb_list, int *__restrict__ fb_count) {
  using Cfg = TileCfg<T>;
  constexpr int TT = Cfg::TT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag, s_nk, s_ng, s_nu;
  TileCta<T, KEEPZ> c;
  c.A = A; c.B = B; c.Add = Add; c.Out = Out;
  c.alpha = alpha; c.beta = beta; c.tau = tau; c.use_add = use_add;
  c.bv = bv; c.up = up; c.rowstat = rowstat;
  c.acc = reinterpret_cast<T *>(smem);
  c.gent = reinterpret_cast<uint4 *>(smem + Cfg::ACC_BYTES);
  c.kkey = reinterpret_cast<int *>(smem + Cfg::ACC_BYTES + Cfg::GENT_BYTES);
  c.kst = c.kkey + Cfg::KT;
  c.gorder = reinterpret_cast<int *>(smem + Cfg::ACC_BYTES + Cfg::GENT_BYTES + Cfg::KTAB_BYTES);
  c.sortbuf = reinterpret_cast<unsigned long long *>(smem + Cfg::ACC_BYTES + Cfg::GENT_BYTES + Cfg::KTAB_BYTES +
                                                     Cfg::ORDER_BYTES);
  c.s_flag = &s_flag; c.s_nk = &s_nk; c.s_ng = &s_ng; c.s_nu = &s_nu;
  c.lane = threadIdx.x & 31;
  c.w = threadIdx.x >> 5;
  c.ncol = Out.n;
  c.lt = lanemask_lt();
  c.wmax = 0;
  c.wover = 0;

  const T cl = c.clean();
  for (int i = threadIdx.x; i < Cfg::SLOTS; i += blockDim.x) c.acc[i] = cl;
  __syncthreads();

  // all tiles, or the tiles of a device-side list (those the split passes could not hold)
  const int ntiles = tile_list ? *((volatile const int *)tile_count) : (A.n + TT - 1) / TT;
  for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
    const int tile = tile_list ? tile_list[q] : q;
    const int end = min(A.n, (tile + 1) * TT);
    int pos = tile * TT, size = first_rows;
    while (pos < end) {
      const int cnt = min(size, end - pos);
      const bool ok = c.process(pos, cnt);
      __syncthreads();  // the tables and the row accumulators are free for the next sub-tile
      if (ok) {
        pos += cnt;
      } else if (cnt > 1) {
        size = cnt / 2;
      } else {  // one row that does not fit: the deferred-row bins take it
        if (threadIdx.x == 0) {
          bool act = true;
          if (bv.row_mat) act = bv.active[bv.row_mat[pos]] != 0;
          if (act) fb_list[atomicAdd(fb_count, 1)] = pos;
        }
        pos += 1;
      }
    }
  }
  if (c.lane == 0) {
    if (c.wmax) atomicMax(&ctl->max_count, c.wmax);
    if (c.wover) atomicAdd(&ctl->overflow_rows, c.wover);
  }
}


// ------------------------------------------------------------------ split form
// The same tiles in two kernels, so that neither waits on the other's phases: a build pass
// (many small CTAs, latency hidden by occupancy) writes per tile the sorted column list U,
// and for every source row the tile reads, its entries' positions in U (16-bit); the
// product pass then needs no table at all: per entry one 16-bit load, the value, and the
// read-modify-write of the row's accumulator.  Tiles are processed in waves so that the
// per-tile records stay small; a tile whose records do not fit goes to the fused kernel.
constexpr int kBuildWarps = 4;
constexpr int kWaveTiles = 8192;
constexpr long long kStagePerTile = 30000;  // mean staged entries a wave's buffer holds per tile

// Records of one wave of tiles (device scratch).
struct TileRecs {
  int *nu;                      // [wave tiles] |U|, or -1: not built (the fused kernel takes the tile)
  int *ucol;                    // [wave tiles][CU] U's columns in order
  unsigned short *stage;        // positions in U of the staged entries of every tile
  long long stage_cap;          // entries `stage` holds
  unsigned long long *cursor;   // next free entry of `stage`
  int *amap;                    // [wave tiles * TT][A.w]: staging index of entry t of a row's source row, minus
                                // the entry's position in that source row
  int *ovf;                     // tiles not built, by global index
  int *ovf_count;
};

template <typename T>
__global__ void __launch_bounds__(kBuildWarps * 32, 8)
    spgemm_tile_build_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, int use_add, BatchView bv, Upper up,
                             int ncol, int tile0, int nwave, TileRecs rec) {
  using Cfg = TileCfg<T>;
  constexpr int TT = Cfg::TT, GT = Cfg::GT, KT = Cfg::KT;
  __shared__ uint4 gent[GT];
  __shared__ int kkey[KT], kst[KT], koff[KT];
  __shared__ int klist[Cfg::MAXK];
  __shared__ int gorder[Cfg::MAXG];
  __shared__ unsigned long long sortbuf[Cfg::MAXG];
  __shared__ int s_flag, s_nk, s_ng, s_nu, s_cnt, s_total;
  __shared__ long long s_base;
  TileCta<T, false> c;
  c.A = A; c.B = B; c.Add = Add;
  c.use_add = use_add; c.bv = bv; c.up = up;
  c.gent = gent; c.kkey = kkey; c.kst = kst; c.gorder = gorder; c.sortbuf = sortbuf;
  c.s_flag = &s_flag; c.s_nk = &s_nk; c.s_ng = &s_ng; c.s_nu = &s_nu;
  c.lane = threadIdx.x & 31;
  c.w = threadIdx.x >> 5;
  c.ncol = ncol;
  c.lt = lanemask_lt();
  const int lane = c.lane, w = c.w;

  for (int t = blockIdx.x; t < nwave; t += gridDim.x) {
    const int tile = tile0 + t;
    const int r0 = tile * TT, nr = min(TT, A.n - r0);
    for (int e = threadIdx.x; e < GT; e += blockDim.x) gent[e] = make_uint4(kNoGroup, 0u, 0u, 0u);
    for (int e = threadIdx.x; e < KT; e += blockDim.x) { kkey[e] = -1; kst[e] = INT_MAX; }
    if (threadIdx.x == 0) { s_flag = 0; s_nk = 0; s_ng = 0; s_nu = 0; }
    __syncthreads();
    // 1. source rows of the tile, each with the first position any row reads
    for (int lr = w; lr < nr; lr += kBuildWarps) {
      const int r = r0 + lr;
      if (bv.row_mat && !bv.active[bv.row_mat[r]]) continue;
      const int na = min(A.nnz[r], A.w);
      for (int s0 = 0; s0 < na; s0 += 32) {
        const int sidx = s0 + lane;
        if (sidx >= na) continue;
        const int k = __ldg(A.idx + (size_t)r * A.w + sidx);
        if ((unsigned)k >= (unsigned)B.n) continue;
        int st = 0;
        if (up.tp) st = min(max(__ldg(up.tp + (size_t)r * A.w + sidx), 0), min(__ldg(B.nnz + k), B.w));
        int h = khash(k, Cfg::LOG2KT), slot = -1;
#pragma unroll 1
        for (int p = 0; p < KT; ++p) {
          const int cur = *((volatile int *)&kkey[h]);
          if (cur == k) { slot = h; break; }
          if (cur == -1) {
            const int old = atomicCAS(&kkey[h], -1, k);
            if (old == -1) { atomicAdd(&s_nk, 1); slot = h; break; }
            if (old == k) { slot = h; break; }
          }
          h = (h + 1) & (KT - 1);
        }
        if (slot >= 0) atomicMin(&kst[slot], st);
        else s_flag = 1;
      }
    }
    __syncthreads();
    bool ok = !s_flag && s_nk <= Cfg::MAXK;
    // 2. the source rows in slot order, their staged lengths and offsets (one warp)
    if (ok && w == 0) {
      int cnt = 0;
      for (int c0 = 0; c0 < KT; c0 += 32) {
        const bool used = kkey[c0 + lane] != -1;
        const unsigned m = __ballot_sync(kFull, used);
        if (used) klist[cnt + __popc(m & c.lt)] = c0 + lane;
        cnt += __popc(m);
      }
      __syncwarp();
      int run = 0;
      for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        int len = 0, slot = 0;
        if (e < cnt) {
          slot = klist[e];
          const int k = kkey[slot];
          len = max(min(__ldg(B.nnz + k), B.w) - kst[slot], 0);
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        if (e < cnt) koff[slot] = run + incl - len;
        run += __shfl_sync(kFull, incl, 31);
      }
      if (lane == 0) {
        s_cnt = cnt;
        s_total = run;
        const unsigned long long b = run > 0 ? atomicAdd(rec.cursor, (unsigned long long)run) : 0ull;
        s_base = (long long)b;
        if ((long long)b + run > rec.stage_cap) s_flag = 1;
      }
    }
    __syncthreads();
    ok = ok && !s_flag;
    const int cnt = s_cnt;
    // 3. U: the staged entries' columns and the addend rows' columns
    if (ok) {
      for (int e = w; e < cnt; e += kBuildWarps) {
        const int slot = klist[e], k = kkey[slot];
        const int nb = min(__ldg(B.nnz + k), B.w);
        const int *bi = B.idx + (size_t)k * B.w;
        for (int q0 = kst[slot]; q0 < nb; q0 += 32) {
          const int q = q0 + lane;
          const int j = q < nb ? __ldg(bi + q) : -1;
          c.insert_col((unsigned)j < (unsigned)ncol, j);
        }
      }
      for (int lr = w; lr < nr; lr += kBuildWarps) {
        const int r = r0 + lr;
        bool add_r = use_add != 0;
        if (bv.row_mat) {
          const int m = bv.row_mat[r];
          add_r = bv.active[m] && bv.beta[m] != 0.0;
        }
        if (!add_r) continue;
        const int nc = min(Add.nnz[r], Add.w);
        const int d0 = up.tpd ? min(max(up.tpd[r], 0), nc) : 0;
        for (int q0 = d0; q0 < nc; q0 += 32) {
          const int q = q0 + lane;
          const int j = q < nc ? Add.idx[(size_t)r * Add.w + q] : -1;
          c.insert_col((unsigned)j < (unsigned)ncol, j);
        }
      }
    }
    __syncthreads();
    ok = ok && !s_flag && s_ng <= Cfg::MAXG;
    // 4. sorted groups and their ranks (one warp)
    if (ok && w == 0) {
      int gc = 0;
      for (int c0 = 0; c0 < GT; c0 += 32) {
        const unsigned gk = gent[c0 + lane].x;
        const bool used = gk != kNoGroup;
        const unsigned m = __ballot_sync(kFull, used);
        if (used) sortbuf[gc + __popc(m & c.lt)] = ((unsigned long long)gk << 32) | (unsigned)(c0 + lane);
        gc += __popc(m);
      }
      __syncwarp();
      if (gc <= 32) c.template rank_groups<1>(gc);
      else if (gc <= 64) c.template rank_groups<2>(gc);
      else if (gc <= 128) c.template rank_groups<4>(gc);
      else c.template rank_groups<8>(gc);
    }
    __syncthreads();
    ok = ok && s_nu <= Cfg::CU;
    if (!ok) {
      if (threadIdx.x == 0) {
        rec.nu[t] = -1;
        rec.ovf[atomicAdd(rec.ovf_count, 1)] = tile;
      }
      __syncthreads();
      continue;
    }
    // 5. U's columns in order
    int *ucol = rec.ucol + (size_t)t * Cfg::CU;
    const int ng = s_ng;
    for (int p = w; p < ng; p += kBuildWarps) {
      const uint4 e = gent[gorder[p]];
      if ((e.y >> lane) & 1u) ucol[(int)e.z + __popc(e.y & c.lt)] = (int)(e.x << 5) + lane;
    }
    // 6. positions in U of every staged entry
    const long long base = s_base;
    for (int e = w; e < cnt; e += kBuildWarps) {
      const int slot = klist[e], k = kkey[slot];
      const int nb = min(__ldg(B.nnz + k), B.w), k0 = kst[slot];
      const int *bi = B.idx + (size_t)k * B.w;
      unsigned short *dst = rec.stage + base + koff[slot] - k0;
      for (int q = k0 + lane; q < nb; q += 32) {
        const int j = __ldg(bi + q);
        const int u = (unsigned)j < (unsigned)ncol ? c.lookup(j) : -1;
        dst[q] = (unsigned short)(u >= 0 ? u : 0xFFFF);
      }
    }
    // 7. per entry of the tile's rows: the staging index of its source row's entries
    for (int lr = w; lr < nr; lr += kBuildWarps) {
      const int r = r0 + lr;
      const int na = min(A.nnz[r], A.w);
      int *am = rec.amap + ((size_t)t * TT + lr) * A.w;
      for (int sidx = lane; sidx < na; sidx += 32) {
        const int k = __ldg(A.idx + (size_t)r * A.w + sidx);
        int v = 0;
        if ((unsigned)k < (unsigned)B.n) {
          int h = khash(k, Cfg::LOG2KT);
#pragma unroll 1
          for (int p = 0; p < KT && kkey[h] != k; ++p) h = (h + 1) & (KT - 1);
          if (kkey[h] == k) v = (int)(base + koff[h] - kst[h]);
        }
        am[sidx] = v;
      }
    }
    if (threadIdx.x == 0) rec.nu[t] = s_nu;
    __syncthreads();
  }
}

// The read-modify-writes of the NU occupied register slots of one source row (a
// predicated-off FP64 instruction still takes its turn in the narrow FP64 pipe, so empty
// slots are not issued at all); slot positions >= CU mark entries outside the product.
template <typename T, bool KEEPZ, int NU, int QW, int CU>
__device__ __forceinline__ void rmw_slots(T *racc, const int (&ur)[QW], const T (&vr)[QW], T a) {
  T old[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u) old[u] = ur[u] < CU ? racc[ur[u]] : T(0);
#pragma unroll
  for (int u = 0; u < NU; ++u)
    if (ur[u] < CU) {
      const T o = (KEEPZ && is_untouched(old[u])) ? T(0) : old[u];
      racc[ur[u]] = fmadd(a, vr[u], o);
    }
}

template <typename T, bool KEEPZ>
__global__ void __launch_bounds__(TileCfg<T>::TT * 32, 2)
    spgemm_tile_apply_kernel(EllView<T> A, EllView<T> B, EllView<T> Add, EllOut<T> Out, T alpha, T beta, T tau,
                             int use_add, BatchView bv, Upper up, int tile0, int nwave, TileRecs rec,
                             double2 *__restrict__ rowstat, SpgemmCtl *__restrict__ ctl) {
  using Cfg = TileCfg<T>;
  constexpr int TT = Cfg::TT, CU = Cfg::CU, QW = Cfg::QW;
  extern __shared__ __align__(16) unsigned char smem[];
  T *acc = reinterpret_cast<T *>(smem);
  int *s_ucol = reinterpret_cast<int *>(smem + Cfg::ACC_BYTES);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int ncol = Out.n;
  const T clean = KEEPZ ? untouched<T>() : T(0);
  const auto tb = mag_bits(tau);
  int wmax = 0, wover = 0;
  for (int i = threadIdx.x; i < TT * CU; i += blockDim.x) acc[i] = clean;
  T *racc = acc + (size_t)w * CU;

  for (int t = blockIdx.x; t < nwave; t += gridDim.x) {
    const int nu = rec.nu[t];
    if (nu < 0) continue;  // the fused kernel takes this tile
    __syncthreads();       // the previous tile's rows are done with s_ucol
    const int *ucol = rec.ucol + (size_t)t * CU;
    for (int i = threadIdx.x; i < nu; i += blockDim.x) s_ucol[i] = ucol[i];
    __syncthreads();
    const int r = (tile0 + t) * TT + w;
    if (r >= A.n) continue;
    T alpha_r = alpha, beta_r = beta;
    int add_r = use_add;
    if (bv.row_mat) {
      const int m = bv.row_mat[r];
      if (!bv.active[m]) continue;
      alpha_r = (T)bv.alpha[m];
      beta_r = (T)bv.beta[m];
      add_r = beta_r != T(0);
    }
    // the addend: positions by binary search in U
    if (add_r) {
      const int nc = min(Add.nnz[r], Add.w);
      const int d0 = up.tpd ? min(max(up.tpd[r], 0), nc) : 0;
      for (int q0 = d0; q0 < nc; q0 += 32) {
        const int q = q0 + lane;
        if (q < nc) {
          const int j = Add.idx[(size_t)r * Add.w + q];
          int lo = 0, hi = nu;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_ucol[mid] < j) lo = mid + 1; else hi = mid;
          }
          if (lo < nu && s_ucol[lo] == j) {
            T o = racc[lo];
            if (KEEPZ && is_untouched(o)) o = T(0);
            racc[lo] = fmadd(beta_r, Add.val[(size_t)r * Add.w + q], o);
          }
        }
      }
      __syncwarp();
    }
    // the source rows in A's order: staged positions, values, read-modify-write
    const int na = min(A.nnz[r], A.w);
    const int *arow_i = A.idx + (size_t)r * A.w;
    const T *arow_v = A.val + (size_t)r * A.w;
    const int *am = rec.amap + ((size_t)t * TT + w) * A.w;
    int ck = 0, cnb = 0, cst = 0, cam = 0, nk_ = 0, nnb = 0, nst = 0, nam = 0;
    T ca = T(0), na_ = T(0);
    auto load_chunk = [&](int cb, int &kk, int &nbk, T &av, int &st, int &amv) {
      const int sidx = cb + lane;
      kk = 0; nbk = 0; av = T(0); st = 0; amv = 0;
      if (sidx < na) {
        const int k = __ldg(arow_i + sidx);
        if ((unsigned)k < (unsigned)B.n) {
          kk = k;
          av = alpha_r * __ldg(arow_v + sidx);
          nbk = min(__ldg(B.nnz + k), B.w);
          if (up.tp) st = min(max(__ldg(up.tp + (size_t)r * A.w + sidx), 0), nbk);
          nbk -= st;
          amv = __ldg(am + sidx) + st;
        }
      }
    };
    load_chunk(0, ck, cnb, ca, cst, cam);
    load_chunk(32, nk_, nnb, na_, nst, nam);
    int cbase = 0;
    auto fetch_step = [&](int tt, int (&ur)[QW], T (&vr)[QW], int &nb, T &a) {
      int k, st, amv;
      if (tt < cbase + 32) {
        k = __shfl_sync(kFull, ck, tt & 31);
        nb = __shfl_sync(kFull, cnb, tt & 31);
        a = __shfl_sync(kFull, ca, tt & 31);
        st = __shfl_sync(kFull, cst, tt & 31);
        amv = __shfl_sync(kFull, cam, tt & 31);
      } else {
        k = __shfl_sync(kFull, nk_, tt & 31);
        nb = __shfl_sync(kFull, nnb, tt & 31);
        a = __shfl_sync(kFull, na_, tt & 31);
        st = __shfl_sync(kFull, nst, tt & 31);
        amv = __shfl_sync(kFull, nam, tt & 31);
      }
      const T *bv_ = B.val + (size_t)k * B.w + st;
      const unsigned short *us = rec.stage + amv;
#pragma unroll
      for (int u = 0; u < QW; ++u) {
        const int q = 32 * u + lane;
        ur[u] = q < nb ? (int)__ldg(us + q) : 0xFFFF;
        vr[u] = q < nb ? __ldg(bv_ + q) : T(0);
      }
      // entries past the registers are read in the step itself
      return 0;
    };
    int u0[QW], u1[QW], u2[QW];
    T v0[QW], v1[QW], v2[QW];
    int nb0 = 0, nb1 = 0, nb2 = 0, am0 = 0, am1 = 0, am2 = 0;
    size_t bo0 = 0, bo1 = 0, bo2 = 0;
    T a0 = T(0), a1 = T(0), a2 = T(0);
    auto info_long = [&](int tt, int &amv, size_t &bo) {  // staging and value offsets of step tt
      int k, st;
      if (tt < cbase + 32) {
        k = __shfl_sync(kFull, ck, tt & 31); st = __shfl_sync(kFull, cst, tt & 31);
        amv = __shfl_sync(kFull, cam, tt & 31);
      } else {
        k = __shfl_sync(kFull, nk_, tt & 31); st = __shfl_sync(kFull, nst, tt & 31);
        amv = __shfl_sync(kFull, nam, tt & 31);
      }
      bo = (size_t)k * B.w + st;
    };
    auto step = [&](const int (&ur)[QW], const T (&vr)[QW], int nb, T a, int amv, size_t bo) {
      switch (min((nb + 31) >> 5, QW)) {
        case 0: break;
        case 1: rmw_slots<T, KEEPZ, 1, QW, CU>(racc, ur, vr, a); break;
        case 2: rmw_slots<T, KEEPZ, 2, QW, CU>(racc, ur, vr, a); break;
        case 3: rmw_slots<T, KEEPZ, 3, QW, CU>(racc, ur, vr, a); break;
        default: rmw_slots<T, KEEPZ, QW, QW, CU>(racc, ur, vr, a); break;
      }
      for (int q = 32 * QW + lane; q < nb; q += 32) {  // source rows longer than the registers
        const int uu = (int)__ldg(rec.stage + amv + q);
        if (uu < CU) {
          T o = racc[uu];
          if (KEEPZ && is_untouched(o)) o = T(0);
          racc[uu] = fmadd(a, __ldg(B.val + bo + q), o);
        }
      }
      __syncwarp();
    };
    if (na > 0) { fetch_step(0, u0, v0, nb0, a0); info_long(0, am0, bo0); }
    if (na > 1) { fetch_step(1, u1, v1, nb1, a1); info_long(1, am1, bo1); }
    for (int tt = 0; tt < na; tt += 3) {
      if (tt >= cbase + 32) {
        ck = nk_; cnb = nnb; ca = na_; cst = nst; cam = nam;
        cbase += 32;
        load_chunk(cbase + 32, nk_, nnb, na_, nst, nam);
      }
      if (tt + 2 < na) { fetch_step(tt + 2, u2, v2, nb2, a2); info_long(tt + 2, am2, bo2); }
      step(u0, v0, nb0, a0, am0, bo0);
      if (tt + 1 >= na) break;
      if (tt + 3 < na) { fetch_step(tt + 3, u0, v0, nb0, a0); info_long(tt + 3, am0, bo0); }
      step(u1, v1, nb1, a1, am1, bo1);
      if (tt + 2 >= na) break;
      if (tt + 4 < na) { fetch_step(tt + 4, u1, v1, nb1, a1); info_long(tt + 4, am1, bo1); }
      step(u2, v2, nb2, a2, am2, bo2);
    }
    // epilogue: U in column order
    int nk = 0;
    double dsum = 0.0, fsum = 0.0;
    int *oi = Out.idx + (size_t)r * Out.w;
    T *ov = Out.val + (size_t)r * Out.w;
    for (int u00 = 0; u00 < nu; u00 += 32) {
      const int u = u00 + lane;
      bool keep = false;
      T v = T(0);
      int j = 0;
      if (u < nu) {
        v = racc[u];
        keep = KEEPZ ? !is_untouched(v) : mag_bits(v) > tb;
        racc[u] = clean;
        j = s_ucol[u];
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
    (void)ncol;
  }
  if (lane == 0) {
    if (wmax) atomicMax(&ctl->max_count, wmax);
    if (wover) atomicAdd(&ctl->overflow_rows, wover);
  }
}

}  // namespace

template <typename T>
int launch_tile(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s) {
  using Cfg = TileCfg<T>;
  constexpr int TT = Cfg::TT, CU = Cfg::CU;
  constexpr int APPLY_SMEM = Cfg::ACC_BYTES + CU * 4;
  const bool keepz = a.tau == 0.0;
  auto fused = keepz ? spgemm_tile_kernel<T, true> : spgemm_tile_kernel<T, false>;
  auto apply = keepz ? spgemm_tile_apply_kernel<T, true> : spgemm_tile_apply_kernel<T, false>;
  static DeviceOnce once_f[2], once_a[2], once_b;
  const int dev = current_device(), kz = keepz ? 1 : 0;
  SP2_TRY(device_once(once_f[kz], dev, [&](int &occ) {
    SP2_CUDA(cudaFuncSetAttribute(fused, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fused, TT * 32, Cfg::SMEM));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  SP2_TRY(device_once(once_a[kz], dev, [&](int &occ) {
    SP2_CUDA(cudaFuncSetAttribute(apply, cudaFuncAttributeMaxDynamicSharedMemorySize, APPLY_SMEM));
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, apply, TT * 32, APPLY_SMEM));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  SP2_TRY(device_once(once_b, dev, [&](int &occ) {
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spgemm_tile_build_kernel<T>, kBuildWarps * 32, 0));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  const int n = a.A->n, aw = a.A->width;
  const int ntiles = (n + TT - 1) / TT;
  const int wave = ntiles < kWaveTiles ? ntiles : kWaveTiles;
  // records of one wave
  auto a256 = [](size_t b) { return ((b + 255) / 256) * 256; };
  const long long stage_cap = (long long)wave * kStagePerTile;
  const size_t b_nu = a256(sizeof(int) * (size_t)wave), b_ucol = a256(sizeof(int) * (size_t)wave * CU);
  const size_t b_stage = a256(sizeof(unsigned short) * (size_t)stage_cap), b_cur = 256;
  const size_t b_amap = a256(sizeof(int) * (size_t)wave * TT * aw), b_ovf = a256(sizeof(int) * ((size_t)wave + 1));
  unsigned char *scr = nullptr;
  SP2_TRY(dev_alloc((void **)&scr, b_nu + b_ucol + b_stage + b_cur + b_amap + b_ovf, s));
  TileRecs rec;
  size_t off = 0;
  rec.nu = reinterpret_cast<int *>(scr + off); off += b_nu;
  rec.ucol = reinterpret_cast<int *>(scr + off); off += b_ucol;
  rec.stage = reinterpret_cast<unsigned short *>(scr + off); off += b_stage;
  rec.stage_cap = stage_cap;
  rec.cursor = reinterpret_cast<unsigned long long *>(scr + off); off += b_cur;
  rec.amap = reinterpret_cast<int *>(scr + off); off += b_amap;
  rec.ovf = reinterpret_cast<int *>(scr + off);
  rec.ovf_count = rec.ovf + wave;
  const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
  const int use_add = a.Add != nullptr && a.beta != 0.0;
  const int first_rows = a.up.tp ? TT : TT / 2;
  const int sms = num_sms();
  int rc = SP2_OK;
  prof_begin(SP2_PROF_SPGEMM, s);
  for (int tile0 = 0; tile0 < ntiles && rc == SP2_OK; tile0 += wave) {
    const int nw = ntiles - tile0 < wave ? ntiles - tile0 : wave;
    cudaError_t e = cudaMemsetAsync(rec.cursor, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rec.ovf_count, 0, sizeof(int), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "row-tile records", __FILE__, __LINE__); break; }
    const int gb = nw < sms * once_b.value[dev] ? nw : sms * once_b.value[dev];
    spgemm_tile_build_kernel<T><<<gb, kBuildWarps * 32, 0, s>>>(view<T>(a.A), view<T>(a.B), add, use_add, a.bv, a.up,
                                                               a.Out->n, tile0, nw, rec);
    note_launch();
    const int ga = nw < sms * once_a[kz].value[dev] ? nw : sms * once_a[kz].value[dev];
    apply<<<ga, TT * 32, APPLY_SMEM, s>>>(view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha, (T)a.beta,
                                          (T)a.tau, use_add, a.bv, a.up, tile0, nw, rec, rowstat, ctl);
    note_launch();
    // tiles whose records did not fit: the fused kernel, which splits them as needed
    const int gf = sms * once_f[kz].value[dev];
    fused<<<gf, TT * 32, Cfg::SMEM, s>>>(view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha, (T)a.beta,
                                         (T)a.tau, use_add, a.bv, a.up, first_rows / 2, rec.ovf, rec.ovf_count,
                                         rowstat, ctl, fb, fb_count);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "row-tile kernels", __FILE__, __LINE__);
  }
  prof_end(SP2_PROF_SPGEMM, s);
  dev_free(scr, s);
  return rc;
}

template int launch_tile<double>(const MultiplyArgs &, double2 *, SpgemmCtl *, int *, int *, cudaStream_t);
template int launch_tile<float>(const MultiplyArgs &, double2 *, SpgemmCtl *, int *, int *, cudaStream_t);

}  // namespace sp2
