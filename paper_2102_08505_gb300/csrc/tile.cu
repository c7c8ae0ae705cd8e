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
                       int use_add, BatchView bv, Upper up, int first_rows, double2 *__restrict__ rowstat,
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

  const int ntiles = (A.n + TT - 1) / TT;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
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

}  // namespace

template <typename T>
int launch_tile(const MultiplyArgs &a, double2 *rowstat, SpgemmCtl *ctl, int *fb, int *fb_count, cudaStream_t s) {
  using Cfg = TileCfg<T>;
  const bool keepz = a.tau == 0.0;
  auto kern = keepz ? spgemm_tile_kernel<T, true> : spgemm_tile_kernel<T, false>;
  static DeviceOnce once[2];
  const int dev = current_device();
  SP2_TRY(device_once(once[keepz ? 1 : 0], dev, [&](int &occ) {
    SP2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
    occ = 0;
    SP2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, Cfg::TT * 32, Cfg::SMEM));
    if (occ < 1) occ = 1;
    return SP2_OK;
  }));
  const long long cap = (long long)num_sms() * once[keepz ? 1 : 0].value[dev];
  const long long tiles = ((long long)a.A->n + Cfg::TT - 1) / Cfg::TT;
  int grid = (int)(tiles < cap ? tiles : cap);
  if (grid < 1) grid = 1;
  // full rows reach about twice the columns of upper-triangle rows: start at half tiles
  const int first_rows = a.up.tp ? Cfg::TT : Cfg::TT / 2;
  const EllView<T> add = a.Add ? view<T>(a.Add) : view<T>(a.A);
  prof_begin(SP2_PROF_SPGEMM, s);
  kern<<<grid, Cfg::TT * 32, Cfg::SMEM, s>>>(view<T>(a.A), view<T>(a.B), add, outview<T>(a.Out), (T)a.alpha,
                                            (T)a.beta, (T)a.tau, a.Add != nullptr && a.beta != 0.0, a.bv, a.up,
                                            first_rows, rowstat, ctl, fb, fb_count);
  note_launch();
  prof_end(SP2_PROF_SPGEMM, s);
  SP2_CUDA(cudaGetLastError());
  return SP2_OK;
}

template int launch_tile<double>(const MultiplyArgs &, double2 *, SpgemmCtl *, int *, int *, cudaStream_t);
template int launch_tile<float>(const MultiplyArgs &, double2 *, SpgemmCtl *, int *, int *, cudaStream_t);

}  // namespace sp2
