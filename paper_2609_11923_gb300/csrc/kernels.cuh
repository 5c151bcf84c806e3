// kernels.cuh — sm_103a kernels of one CFR+ iteration over the compiled game.
//
// Stage (a), forward reach (eq. (opfwd) on both lanes, eq. (lanes)): reach
//   is stored for internal nodes only (terminal reach is never read), by
//   internal rank. Member order (the default): each thread takes four
//   internal nodes of depth d + 1, and each reads its parent's reach through
//   its edge record and writes its own (fwd_pull). Breadth-first and
//   value-slot orders: each thread takes four internal nodes of depth d and
//   writes both reach lanes of their internal children (fwd_int4). The
//   acting player's lane is multiplied by sigma(I, a); the other lane and
//   chance edges copy through (the paper's sentinel multiplier 1 becomes a
//   branch on the edge's slot word).
// Stage (b), terminal utility: the value array holds pi_c(z) u(z) in every
//   terminal's value slot from bind time on (eq. (template)); no kernel
//   writes it again, which removes the per-iteration template copy.
// Stages (c) + (d), backward (eqs. (opbwd), (instregret), (regret), (rm)):
//   values live in value slots: the children of one set's members form one
//   contiguous block, and every node writes its own value into its parent's
//   block. Per depth, chance nodes sum their children's values (one thread
//   each; a chance root is skipped, nothing reads its value) and every
//   information set of that depth is handled by one group of LANES lanes,
//   which reads its members' reach as one run in member order: members' values v(h) = sum_a sigma(I,a) v(h.a), the regret terms
//   s * pi_{-i}(h) * (v(h.a) - v(h)) and the average terms pi_i(h) sigma(I,a)
//   are summed over members in a fixed order (no atomics), then
//   R <- max(R + r, 0) (CFR+), avg += t * m, and sigma^{t+1}(I,.) = RM(R) is
//   written in place (nothing reads sigma(I,.) again in this iteration).
//   P64 sums members strictly in ascending node order (lane order within each
//   chunk of LANES members), the order of the recursive definition; P32 keeps
//   per-lane partial sums and finishes with an xor butterfly (fixed shape,
//   deterministic run to run).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cfr {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using vec2_t = typename Vec2<T>::type;

constexpr int kThreads = 256;
constexpr int32_t kP2Bit = 1 << 30;
constexpr int32_t kMask = kP2Bit - 1;

// Loads of arrays that a persistent kernel rewrites between grid barriers go
// around L1 (ld.global.cg): L1 is not coherent across SMs.
template <bool PERSIST, typename X>
__device__ __forceinline__ X ldm(const X *p) {
  if constexpr (PERSIST) return __ldcg(p);
  else return *p;
}

// Programmatic dependent launch between the per-level kernels: every such
// kernel first waits until the launch before it has completed and its
// writes are visible (griddepcontrol.wait; a no-op without a programmatic
// dependency), then lets the next launch start being scheduled
// (launch_dependents), so the next kernel's launch and block scheduling
// overlap this kernel's tail instead of following it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

constexpr int32_t kWideNode = 1024;   // chance nodes above this fan-out go by chunks
constexpr int32_t kWideChunkK = 2048; // children per chunk of a wide node

struct GameView {
  const int32_t *__restrict__ iset_slot;
  const int32_t *__restrict__ iset_mem;
  // value slots: a set's members' children form one block starting at
  // iset_vb[I] (action-major: child a of member k at iset_vb[I] + a * M +
  // (k - first member), M members); every node writes its own value to the
  // slot its parent reads (mem_vs, ch_vs, wide_vs)
  const int32_t *__restrict__ iset_vb;
  const int32_t *__restrict__ mem_vs;
  const int32_t *__restrict__ ch_vb;       // narrow chance nodes: children's block,
  const int32_t *__restrict__ ch_nch;      //   child count,
  const int32_t *__restrict__ ch_vs;       //   own value slot
  const int32_t *__restrict__ wide_vb;     // wide chance nodes: the same
  const int32_t *__restrict__ wide_nch;
  const int32_t *__restrict__ wide_vs;
  const int32_t *__restrict__ wide_chunk;  // prefix of their chunk counts
  double *wide_part;                       // [3 * chunks] partial sums
  unsigned *wide_cnt;                      // [wide nodes] chunks finished (reset by the last one)
  // compact index space of the internal nodes (reach is stored only there)
  const int32_t *__restrict__ int_slot;    // slot word of each internal node
  const uint32_t *__restrict__ int_mask;   // internal children (bit a), or kBigBit
  const int32_t *__restrict__ int_cirank;  // rank of the first internal child, or big_irank offset
  const int32_t *__restrict__ big_irank;   // [nch, child ranks...] of nodes with > 31 children
  const int2 *__restrict__ int_edge;       // member order: each internal node's (parent rank, slot word of
                                           //   its edge or -1 under chance); else null
  const int32_t *__restrict__ mem_irank;   // internal rank of each member (null in member order)
  const int2 *__restrict__ iset_rank;      // member order: per set, rank of member 0 and the stride
                                           //   of its members' ranks (else null)
  const int32_t *__restrict__ wide_irank;  // internal rank of each wide node
};

constexpr uint32_t kBigBit = 0x80000000u;

template <typename T> struct StateView {
  vec2_t<T> *reach;
  T *v;
  T *sigma;
  double *R;
  double *avg;
  long long *t;  // completed iterations; iteration t+1 uses weight w = t+1
};

struct LevelWork {
  int32_t ib, ie;         // internal ranks of depth d
  int32_t lb, le;         // nodes of depth d
  int32_t ch0, ch1;       // narrow chance nodes of depth d (ch_* arrays)
  int32_t is0, is2, is1;  // sets of depth d: player 1 [is0, is2), player 2 [is2, is1)
  int32_t wd0, wd1;       // wide chance nodes of depth d (wide_* arrays)
  int32_t wc0, wc1;       // their chunks
  int32_t fan;            // 1 if a chance node of depth d has more than kFanLight internal children
};

// Where set I's members keep their reach: member k (global member index) has
// rank kb + k * rg (member order), or the rank table's entry (kb = rg = 0).
struct MemberRanks {
  int32_t kb, rg;
};

__device__ __forceinline__ MemberRanks member_ranks(const GameView &g, int32_t I, int32_t m0) {
  MemberRanks mr{0, 0};
  if (g.iset_rank) {
    const int2 x = __ldg(g.iset_rank + I);
    mr.rg = x.y;
    mr.kb = x.x - m0 * x.y;
  }
  return mr;
}

// The wide node owning chunk q (binary search over the level's prefix).
__device__ __forceinline__ int32_t wide_of_chunk(const GameView &g, const LevelWork &w, int32_t q) {
  int32_t lo = w.wd0, hi = w.wd1 - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(g.wide_chunk + mid) <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Fixed-shape block reduction (all threads call it; the result is valid in thread 0).
__device__ __forceinline__ double block_sum(double x) {
  __shared__ double sm[kThreads];
  __syncthreads();
  sm[threadIdx.x] = x;
  __syncthreads();
#pragma unroll
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  return sm[0];
}

// The sum of v[cb, ce) strictly left to right (the FP64 parity order), for
// one block of N threads that all call it: the block stages N values at a
// time in shared memory, and thread 0 adds one batch while the others load
// the next. The result is valid in thread 0.
template <int N, bool PERSIST, typename T>
__device__ __forceinline__ double ordered_sum(const T *v, int32_t cb, int32_t ce) {
  __shared__ double buf[2 * N];
  const int tid = threadIdx.x;
  double s = 0.0;
  if (cb + tid < ce) buf[tid] = (double)ldm<PERSIST>(v + cb + tid);
  __syncthreads();
  int b = 0;
  for (int32_t c0 = cb; c0 < ce; c0 += N) {
    if (c0 + N + tid < ce) buf[(b ^ 1) * N + tid] = (double)ldm<PERSIST>(v + c0 + N + tid);
    if (tid == 0) {
      const int n = ce - c0 < N ? ce - c0 : N;
      for (int j = 0; j < n; ++j) s = s + buf[b * N + j];
    }
    __syncthreads();
    b ^= 1;
  }
  return s;
}

// ------------------------------------------------------------ forward reach
// reach of child a of an internal node with slot word s and reach r
template <typename T, bool PERSIST>
__device__ __forceinline__ vec2_t<T> child_reach(const T *sigma, int32_t s, vec2_t<T> r, int a) {
  if (s >= 0) {
    const T sa = ldm<PERSIST>(sigma + (s & kMask) + a);
    if (s & kP2Bit) r.y = r.y * sa;
    else r.x = r.x * sa;
  }
  return r;
}

// Writes the reach of the internal children of one internal node: children
// flagged in the mask get consecutive internal ranks from cir on; nodes with
// more than 31 children list their children's ranks in big_irank (terminal
// children -1, never written: nothing reads a terminal's reach).
template <typename T, bool PERSIST>
__device__ __forceinline__ void fwd_write(const GameView &g, const T *sigma, vec2_t<T> *reach, int32_t s,
                                          uint32_t mask, int32_t cir, vec2_t<T> r) {
  if (mask & kBigBit) {
    const int32_t nch = __ldg(g.big_irank + cir);
    if (nch > kWideNode) return;  // wide: done by chunks
    for (int32_t a = 0; a < nch; ++a) {
      const int32_t q = __ldg(g.big_irank + cir + 1 + a);
      if (q >= 0) reach[q] = child_reach<T, PERSIST>(sigma, s, r, a);
    }
  } else {
    int32_t q = cir;
    while (mask) {
      const int a = __ffs(mask) - 1;
      mask &= mask - 1;
      reach[q++] = child_reach<T, PERSIST>(sigma, s, r, a);
    }
  }
}

constexpr int kFanLight = 4;  // chance nodes with more internal children are written by the whole warp

// Four internal nodes q, q+stride, q+2 stride, q+3 stride per thread: their
// records and reach are read together (coalesced), then their children's
// reach is written. A chance node's internal children all copy its reach, so
// a chance node with many of them (a card dealt mid-game) is written by the
// whole warp as one coalesced run instead of by its own thread alone. All 32
// lanes of the warp call this together (q = warp base + lane; a lane whose
// nodes lie past qe still takes part in the warp-wide writes).
template <typename T, bool PERSIST, bool FAN>
__device__ __forceinline__ void fwd_int4(const GameView &g, const T *sigma, vec2_t<T> *reach, int32_t q,
                                         int32_t stride, int32_t qe) {
  int32_t sl[4], ci[4];
  uint32_t mk[4];
  vec2_t<T> r[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int32_t x = q + u * stride;
    mk[u] = 0u; sl[u] = -1; ci[u] = 0;
    r[u].x = T(0); r[u].y = T(0);
    if (x < qe) {
      sl[u] = __ldg(g.int_slot + x);
      mk[u] = __ldg(g.int_mask + x);
      ci[u] = __ldg(g.int_cirank + x);
      r[u] = ldm<PERSIST>(reach + x);
    }
  }
  if constexpr (!FAN) {  // depths without chance nodes of many internal children
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (mk[u]) fwd_write<T, PERSIST>(g, sigma, reach, sl[u], mk[u], ci[u], r[u]);
    return;
  }
  bool hvy[4], any = false;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    hvy[u] = sl[u] < 0 && mk[u] != 0u && ((mk[u] & kBigBit) || __popc(mk[u]) > kFanLight);
    any = any || hvy[u];
  }
  if (!__any_sync(0xffffffffu, any)) {  // the common case: every node of the warp is light
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (mk[u]) fwd_write<T, PERSIST>(g, sigma, reach, sl[u], mk[u], ci[u], r[u]);
    return;
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const bool heavy = hvy[u];
    unsigned hv = __ballot_sync(0xffffffffu, heavy);
    if (mk[u] && !heavy) fwd_write<T, PERSIST>(g, sigma, reach, sl[u], mk[u], ci[u], r[u]);
    while (hv) {
      const int j = __ffs(hv) - 1;
      hv &= hv - 1;
      const uint32_t m = __shfl_sync(0xffffffffu, mk[u], j);
      const int32_t c0 = __shfl_sync(0xffffffffu, ci[u], j);
      vec2_t<T> rr;
      rr.x = __shfl_sync(0xffffffffu, r[u].x, j);
      rr.y = __shfl_sync(0xffffffffu, r[u].y, j);
      if (m & kBigBit) {
        const int32_t nch = __ldg(g.big_irank + c0);
        if (nch <= kWideNode)  // wide nodes go by chunks
          for (int32_t a = lane; a < nch; a += 32) {
            const int32_t c = __ldg(g.big_irank + c0 + 1 + a);
            if (c >= 0) reach[c] = rr;
          }
      } else {
        const int n = __popc(m);
        for (int i = lane; i < n; i += 32) reach[c0 + i] = rr;
      }
    }
  }
}

// One chunk of a wide chance node: its internal children copy its reach.
template <typename T, bool PERSIST>
__device__ __forceinline__ void fwd_wide_chunk(const GameView &g, const LevelWork &w, vec2_t<T> *reach, int32_t q) {
  const int32_t wi = wide_of_chunk(g, w, q);
  const int32_t ir = __ldg(g.wide_irank + wi);
  const int32_t off = __ldg(g.int_cirank + ir);
  const int32_t nch = __ldg(g.big_irank + off);
  const int32_t j0 = (q - __ldg(g.wide_chunk + wi)) * kWideChunkK;
  const int32_t j1 = min(nch, j0 + kWideChunkK);
  const vec2_t<T> r = ldm<PERSIST>(reach + ir);
  for (int32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int32_t c = __ldg(g.big_irank + off + 1 + j);
    if (c >= 0) reach[c] = r;
  }
}

// Grid: nb_nodes blocks over the internal nodes of depth d, then one block
// per wide chunk.
template <typename T, bool FAN>
__global__ void __launch_bounds__(kThreads) fwd_level_kernel(GameView g, const T *sigma, vec2_t<T> *reach,
                                                            LevelWork w, int nb_nodes) {
  pdl_enter();
  if ((int)blockIdx.x >= nb_nodes) {
    fwd_wide_chunk<T, false>(g, w, reach, w.wc0 + (int32_t)blockIdx.x - nb_nodes);
    return;
  }
  const int32_t stride = nb_nodes * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int32_t qw = w.ib + blockIdx.x * blockDim.x + (threadIdx.x & ~31); qw < w.ie; qw += 4 * stride)
    fwd_int4<T, false, FAN>(g, sigma, reach, qw + lane, stride, w.ie);
}

// Member order: each internal node of ranks [qb, qe) (one depth) pulls its
// reach from its parent's, times the strategy of its edge in the acting
// player's lane (a chance edge copies it). kPull nodes per thread in flight.
constexpr int kPull = 4;
template <typename T, bool PERSIST>
__device__ __forceinline__ void fwd_pull(const GameView &g, const T *sigma, vec2_t<T> *reach, int32_t q,
                                         int32_t stride, int32_t qe) {
  int2 e[kPull];
#pragma unroll
  for (int u = 0; u < kPull; ++u) {
    const int32_t x = q + u * stride;
    e[u] = make_int2(-1, -1);
    if (x < qe) e[u] = __ldg(g.int_edge + x);
  }
  vec2_t<T> r[kPull];
  T sa[kPull];
#pragma unroll
  for (int u = 0; u < kPull; ++u) {
    r[u].x = T(0); r[u].y = T(0);
    sa[u] = T(1);
    if (e[u].x >= 0) {
      r[u] = ldm<PERSIST>(reach + e[u].x);
      if (e[u].y >= 0) sa[u] = ldm<PERSIST>(sigma + (e[u].y & kMask));
    }
  }
#pragma unroll
  for (int u = 0; u < kPull; ++u) {
    if (e[u].x < 0) continue;
    if (e[u].y >= 0) {
      if (e[u].y & kP2Bit) r[u].y = r[u].y * sa[u];
      else r[u].x = r[u].x * sa[u];
    }
    reach[q + u * stride] = r[u];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) fwd_pull_kernel(GameView g, const T *sigma, vec2_t<T> *reach,
                                                            int32_t qb, int32_t qe) {
  pdl_enter();
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t q = qb + blockIdx.x * blockDim.x + threadIdx.x; q < qe; q += kPull * stride)
    fwd_pull<T, false>(g, sigma, reach, q, stride, qe);
}

// ------------------------------------------------------------ group helpers
template <int LANES>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (LANES == 32) return 0xffffffffu;
  else return ((1u << LANES) - 1u) << (((threadIdx.x & 31) / LANES) * LANES);
}

template <int LANES, typename X>
__device__ __forceinline__ X group_sum_butterfly(X x, unsigned mask) {
#pragma unroll
  for (int off = LANES / 2; off > 0; off >>= 1) x += __shfl_xor_sync(mask, x, off, LANES);
  return x;
}

// ------------------------------------------------------------- update rules
// CFR+ clamps the cumulative regret at zero; vanilla CFR does not; PCFR+
// clamps like CFR+ and matches the next strategy against R + r, the
// iteration's instantaneous regret serving as the prediction (Section 3,
// update rules).
constexpr int kRuleCfrPlus = 0, kRuleCfr = 1, kRulePcfrPlus = 2;

// Averaging weight of iteration t (1-based): t, or t^2 under PCFR+.
__device__ __forceinline__ double avg_weight(long long t, int rule) {
  const double x = (double)t;
  return rule == kRulePcfrPlus ? x * x : x;
}

// One slot's update from its set's totals (instantaneous regret r, average
// term m): R <- R + r (clamped at 0 except under vanilla CFR), avg += w * m.
// Returns what regret matching takes the positive part of: the new R, or
// R + r under PCFR+.
__device__ __forceinline__ double slot_update(double *R, double *avg, int32_t q, double r, double m, double wt,
                                              int rule) {
  double Rn = R[q] + r;
  if (rule != kRuleCfr) Rn = Rn > 0.0 ? Rn : 0.0;
  R[q] = Rn;
  avg[q] += wt * m;
  const double x = rule == kRulePcfrPlus ? Rn + r : Rn;
  return x > 0.0 ? x : 0.0;
}

// ------------------------------------------------------------- backward
// Narrow chance node i: the sum of its children's values (left to right).
template <typename T, bool PERSIST>
__device__ __forceinline__ void bwd_chance(const GameView &g, T *v, int32_t i) {
  const int32_t cb = __ldg(g.ch_vb + i), ce = cb + __ldg(g.ch_nch + i);
  T s = T(0);
  for (int32_t c = cb; c < ce; ++c) s = s + ldm<PERSIST>(v + c);
  v[__ldg(g.ch_vs + i)] = s;
}

// One chunk of a wide chance node's value sum. P32: every chunk block sums
// its children (fixed shape), and the block that finishes last adds the
// chunk partials in chunk order (an integer ticket decides who is last; no
// float atomics). P64: the first chunk's block sums all children strictly
// left to right, the order of the recursive definition.
template <typename T, bool PERSIST>
__device__ __forceinline__ void bwd_wide_chunk(const GameView &g, const LevelWork &w, T *v, int32_t q) {
  const int32_t wi = wide_of_chunk(g, w, q);
  const int32_t h = __ldg(g.wide_vs + wi);  // the node's own value slot
  const int32_t cb = __ldg(g.wide_vb + wi), ce = cb + __ldg(g.wide_nch + wi);
  const int32_t q0 = __ldg(g.wide_chunk + wi), nq = __ldg(g.wide_chunk + wi + 1) - q0;
  if constexpr (sizeof(T) == 8) {
    if (q == q0) {  // block-uniform: the whole block stages the children
      const double s = ordered_sum<kThreads, PERSIST>(v, cb, ce);
      if (threadIdx.x == 0) v[h] = s;
    }
    return;
  } else {
    const int32_t c0 = cb + (q - q0) * kWideChunkK, c1 = min(ce, c0 + kWideChunkK);
    double x = 0.0;
    for (int32_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) x += (double)ldm<PERSIST>(v + c);
    x = block_sum(x);
    __shared__ unsigned s_ticket;
    if (threadIdx.x == 0) {
      g.wide_part[q] = x;
      __threadfence();
      s_ticket = atomicAdd(g.wide_cnt + wi, 1u);
    }
    __syncthreads();
    if (s_ticket == (unsigned)(nq - 1)) {  // the last chunk's block adds the partials (fixed shape)
      __threadfence();
      double y = 0.0;
      for (int32_t k = threadIdx.x; k < nq; k += blockDim.x) y += __ldcg(g.wide_part + q0 + k);
      y = block_sum(y);
      if (threadIdx.x == 0) {
        v[h] = (T)y;
        g.wide_cnt[wi] = 0u;
      }
    }
  }
}

// A member's two indices (member order: coalesced reads): its own value slot
// and its internal rank (where its reach lives; in member order the rank
// follows from the member index and the set's rank base and stride). Past
// the set's end: -1.
__device__ __forceinline__ int32_t member_rank(const GameView &g, int32_t k, MemberRanks mr) {
  return g.mem_irank ? __ldg(g.mem_irank + k) : mr.kb + k * mr.rg;
}

__device__ __forceinline__ void member_idx(const GameView &g, int32_t k, int32_t m1, MemberRanks mr, int32_t &ps,
                                           int32_t &ir) {
  ps = -1;
  ir = -1;
  if (k < m1) {
    ps = __ldg(g.mem_vs + k);
    ir = member_rank(g, k, mr);
  }
}

// Loads and per-member terms of one member (k < m1) whose indices are
// already known, or zeros. The member's child a is slot vb + a * M + (k -
// m0) of the set's block (M = m1 - m0 members): for each action the group's
// lanes read consecutive members' children as one run. The average-strategy terms are
// pw * sigma(a). LEAN (FP32 only): only pw is carried (mm[0]) and the set's
// sum of pw is multiplied by sigma(a) once (avg_terms), which frees
// registers where the budget is tight; otherwise each product is added, in
// member order in FP64, as the definition does.
template <typename T, int MAXA, bool PERSIST, bool LEAN = false>
__device__ __forceinline__ void member_data(const GameView &g, const StateView<T> &st, int32_t k, int32_t m0,
                                            int32_t m1, int32_t vb, int32_t na, bool p2, const T (&sig)[MAXA],
                                            int32_t h, int32_t ir, T (&d)[MAXA], T (&mm)[MAXA]) {
#pragma unroll
  for (int a = 0; a < MAXA; ++a) { d[a] = T(0); mm[a] = T(0); }
  if (k >= m1) return;
  const int32_t cb = vb + (k - m0), M = m1 - m0;
  const vec2_t<T> r = ldm<PERSIST>(st.reach + ir);
  T vc[MAXA];
  T vh = T(0);
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    if (a < na) {
      vc[a] = ldm<PERSIST>(st.v + cb + a * M);
      vh = vh + sig[a] * vc[a];
    }
  }
  st.v[h] = vh;
  const T po = p2 ? r.x : r.y;  // opponent's reach (chance is inside v)
  const T pw = p2 ? r.y : r.x;  // own reach
  const T f = (p2 ? T(-1) : T(1)) * po;
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    if (a < na) {
      d[a] = f * (vc[a] - vh);
      if constexpr (!LEAN || sizeof(T) == 8) mm[a] = pw * sig[a];
    }
  }
  if constexpr (LEAN && sizeof(T) == 4) mm[0] = pw;
}

// LEAN FP32: the set's average terms sigma(a) * (sum of the members' own
// reach), from the sum carried in macc[0].
template <typename T, int MAXA>
__device__ __forceinline__ void avg_terms(const T (&sig)[MAXA], int32_t na, T (&macc)[MAXA]) {
  const T spw = macc[0];
#pragma unroll
  for (int a = 0; a < MAXA; ++a) macc[a] = a < na ? sig[a] * spw : T(0);
}

// Indices, loads and per-member terms of one member (k < m1), or zeros.
template <typename T, int MAXA, bool PERSIST, bool LEAN = false>
__device__ __forceinline__ void member_terms(const GameView &g, const StateView<T> &st, int32_t k, int32_t m0,
                                             int32_t m1, MemberRanks mr, int32_t vb, int32_t na, bool p2,
                                             const T (&sig)[MAXA], T (&d)[MAXA], T (&mm)[MAXA]) {
  int32_t h, ir;
  member_idx(g, k, m1, mr, h, ir);
  member_data<T, MAXA, PERSIST, LEAN>(g, st, k, m0, m1, vb, na, p2, sig, h, ir, d, mm);
}

// Adds one chunk's member terms to the group totals. P64: lane order (the
// members' ascending order), every lane ends with the same totals. P32:
// per-lane partial sums (finished by a butterfly).
template <typename T, int MAXA, int LANES>
__device__ __forceinline__ void accumulate_chunk(int32_t cnt, int32_t na, unsigned mask, const T (&d)[MAXA],
                                                 const T (&mm)[MAXA], T (&racc)[MAXA], T (&macc)[MAXA]) {
  if constexpr (sizeof(T) == 8) {
    if constexpr (LANES <= 8) {  // unrolled: the shuffles issue ahead of the ordered adds
#pragma unroll
      for (int j = 0; j < LANES; ++j) {
        if (j < cnt) {
#pragma unroll
          for (int a = 0; a < MAXA; ++a) {
            if (a < na) {
              racc[a] = racc[a] + __shfl_sync(mask, d[a], j, LANES);
              macc[a] = macc[a] + __shfl_sync(mask, mm[a], j, LANES);
            }
          }
        }
      }
    } else {  // wide groups keep the loop (registers)
      for (int j = 0; j < cnt; ++j) {
#pragma unroll
        for (int a = 0; a < MAXA; ++a) {
          if (a < na) {
            racc[a] = racc[a] + __shfl_sync(mask, d[a], j, LANES);
            macc[a] = macc[a] + __shfl_sync(mask, mm[a], j, LANES);
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      racc[a] += d[a];
      macc[a] += mm[a];
    }
  }
}

// One information set, processed by the LANES lanes of one group. Members go
// in chunks of LANES (two chunks per step for narrow groups); each step loads
// the next step's member indices while its own reach and child values are in
// flight, so a step waits for one memory round trip, not two. The update of
// the set's slots runs one lane per action. LEAN: see member_data.
template <typename T, int MAXA, int LANES, bool PERSIST, bool LEAN = false>
__device__ __forceinline__ void bwd_set(const GameView &g, const StateView<T> &st, int32_t I, bool p2,
                                        int lane, unsigned mask, double wt, int rule, int upd) {
  const int32_t sb = __ldg(g.iset_slot + I);
  const int32_t na = __ldg(g.iset_slot + I + 1) - sb;
  const int32_t m0 = __ldg(g.iset_mem + I), m1 = __ldg(g.iset_mem + I + 1);
  const int32_t vb = __ldg(g.iset_vb + I);
  const MemberRanks mr = member_ranks(g, I, m0);
  T sig[MAXA], racc[MAXA], macc[MAXA];
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    sig[a] = a < na ? ldm<PERSIST>(st.sigma + sb + a) : T(0);
    racc[a] = T(0);
    macc[a] = T(0);
  }
  constexpr bool TWO = MAXA <= 8 && LANES <= 8;  // narrow groups keep two chunks in flight
  constexpr int NCH = 2;
  int32_t k0 = m0;
  // The two forms below compute the same; the one with chunk arrays
  // compiles to fewer spills in LEAN kernels (64 registers a thread), the
  // one with named chunks runs faster with a larger register budget.
  if constexpr (TWO && LEAN) {
    if (k0 + (NCH - 1) * LANES < m1) {
      int32_t ps[NCH], ir[NCH];
#pragma unroll
      for (int j = 0; j < NCH; ++j) member_idx(g, k0 + j * LANES + lane, m1, mr, ps[j], ir[j]);
      for (; k0 + (NCH - 1) * LANES < m1; k0 += NCH * LANES) {
        int32_t qs[NCH], jr[NCH];  // the next step's indices
#pragma unroll
        for (int j = 0; j < NCH; ++j) member_idx(g, k0 + (NCH + j) * LANES + lane, m1, mr, qs[j], jr[j]);
        T d[NCH][MAXA], mm[NCH][MAXA];
#pragma unroll
        for (int j = 0; j < NCH; ++j)
          member_data<T, MAXA, PERSIST, LEAN>(g, st, k0 + j * LANES + lane, m0, m1, vb, na, p2, sig, ps[j], ir[j],
                                              d[j], mm[j]);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {  // chunks in member order
          const int32_t left = m1 - k0 - j * LANES;
          accumulate_chunk<T, MAXA, LANES>(left < 0 ? 0 : (left < LANES ? left : LANES), na, mask, d[j], mm[j], racc,
                                           macc);
        }
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          ps[j] = qs[j];
          ir[j] = jr[j];
        }
      }
    }
  } else if constexpr (TWO) {
    if (k0 + LANES < m1) {
      int32_t ps0, ir0, ps1, ir1;
      member_idx(g, k0 + lane, m1, mr, ps0, ir0);
      member_idx(g, k0 + LANES + lane, m1, mr, ps1, ir1);
      for (; k0 + LANES < m1; k0 += 2 * LANES) {
        int32_t qs0, jr0, qs1, jr1;  // the next step's indices
        member_idx(g, k0 + 2 * LANES + lane, m1, mr, qs0, jr0);
        member_idx(g, k0 + 3 * LANES + lane, m1, mr, qs1, jr1);
        T d0[MAXA], mm0[MAXA], d1[MAXA], mm1[MAXA];
        member_data<T, MAXA, PERSIST, LEAN>(g, st, k0 + lane, m0, m1, vb, na, p2, sig, ps0, ir0, d0, mm0);
        member_data<T, MAXA, PERSIST, LEAN>(g, st, k0 + LANES + lane, m0, m1, vb, na, p2, sig, ps1, ir1, d1, mm1);
        accumulate_chunk<T, MAXA, LANES>(LANES, na, mask, d0, mm0, racc, macc);
        const int32_t c1 = (m1 - k0 - LANES) < LANES ? (m1 - k0 - LANES) : LANES;
        accumulate_chunk<T, MAXA, LANES>(c1, na, mask, d1, mm1, racc, macc);
        ps0 = qs0; ir0 = jr0; ps1 = qs1; ir1 = jr1;
      }
    }
  }
  if constexpr (TWO) {  // the last chunk
    for (; k0 < m1; k0 += LANES) {
      T d[MAXA], mm[MAXA];
      member_terms<T, MAXA, PERSIST, LEAN>(g, st, k0 + lane, m0, m1, mr, vb, na, p2, sig, d, mm);
      const int32_t cnt = (m1 - k0) < LANES ? (m1 - k0) : LANES;
      accumulate_chunk<T, MAXA, LANES>(cnt, na, mask, d, mm, racc, macc);
    }
  } else {
    int32_t ps, ir;
    member_idx(g, k0 + lane, m1, mr, ps, ir);
    for (; k0 < m1; k0 += LANES) {
      int32_t qs, jr;  // the next step's indices
      member_idx(g, k0 + LANES + lane, m1, mr, qs, jr);
      T d[MAXA], mm[MAXA];
      member_data<T, MAXA, PERSIST, LEAN>(g, st, k0 + lane, m0, m1, vb, na, p2, sig, ps, ir, d, mm);
      const int32_t cnt = (m1 - k0) < LANES ? (m1 - k0) : LANES;
      accumulate_chunk<T, MAXA, LANES>(cnt, na, mask, d, mm, racc, macc);
      ps = qs; ir = jr;
    }
  }
  // alternating updates: the other player's sets only pass their values up
  if (!(upd & (p2 ? 2 : 1))) return;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      if (a < na) {
        racc[a] = group_sum_butterfly<LANES>(racc[a], mask);
        if constexpr (!LEAN) macc[a] = group_sum_butterfly<LANES>(macc[a], mask);
      }
    }
    if constexpr (LEAN) {
      macc[0] = group_sum_butterfly<LANES>(macc[0], mask);
      avg_terms<T, MAXA>(sig, na, macc);
    }
  }
  // every lane now holds the set's totals racc[a], macc[a]
  if (na <= LANES) {
    // lane a updates slot a (slot_update), then sigma^{t+1} = RM; the sum of
    // positive parts runs in action order
    T r = T(0), m = T(0);
#pragma unroll
    for (int a = 0; a < MAXA; ++a)
      if (a == lane) { r = racc[a]; m = macc[a]; }
    double pos = 0.0;
    if (lane < na) pos = slot_update(st.R, st.avg, sb + lane, (double)r, (double)m, wt, rule);
    if constexpr (sizeof(T) == 8) {
      double tot = 0.0;
      for (int a = 0; a < na; ++a) tot += __shfl_sync(mask, pos, a, LANES);
      if (lane < na) st.sigma[sb + lane] = tot > 0.0 ? pos / tot : 1.0 / (double)na;
    } else {
      const float pf = (float)pos;
      float tot = 0.f;
      for (int a = 0; a < na; ++a) tot += __shfl_sync(mask, pf, a, LANES);
      if (lane < na) st.sigma[sb + lane] = tot > 0.f ? pf / tot : 1.f / (float)na;
    }
  } else if (lane == 0) {
    double pos[MAXA];
    double tot = 0.0;
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      if (a < na) {
        pos[a] = slot_update(st.R, st.avg, sb + a, (double)racc[a], (double)macc[a], wt, rule);
        tot += pos[a];
      }
    }
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int a = 0; a < MAXA; ++a)
        if (a < na) st.sigma[sb + a] = tot > 0.0 ? pos[a] / tot : 1.0 / (double)na;
    } else {
      float totf = 0.f;
#pragma unroll
      for (int a = 0; a < MAXA; ++a)
        if (a < na) totf += (float)pos[a];
#pragma unroll
      for (int a = 0; a < MAXA; ++a)
        if (a < na) st.sigma[sb + a] = totf > 0.f ? (float)pos[a] / totf : 1.f / (float)na;
    }
  }
}

// One information set per block, for depths with few sets of hundreds of
// members each: all kThreads threads load members tid, tid + kThreads, ...
// at once. P64: each chunk's member terms are staged in shared memory and
// thread a adds column a in ascending member order, the order the group form
// uses, so the result is bitwise the same; P32: per-thread partial sums
// finished by a fixed-shape tree. The slot update runs one thread per action.
template <typename T, int MAXA>
__device__ __forceinline__ void bwd_set_block(const GameView &g, const StateView<T> &st, int32_t I, bool p2,
                                              double wt, int rule, int upd) {
  __shared__ T s_d[kThreads * MAXA], s_m[kThreads * MAXA];  // [member][action]
  __shared__ double s_pos[MAXA];
  const int tid = threadIdx.x;
  const int32_t sb = __ldg(g.iset_slot + I);
  const int32_t na = __ldg(g.iset_slot + I + 1) - sb;
  const int32_t m0 = __ldg(g.iset_mem + I), m1 = __ldg(g.iset_mem + I + 1);
  const int32_t vb = __ldg(g.iset_vb + I);
  const MemberRanks mr = member_ranks(g, I, m0);
  T sig[MAXA], racc[MAXA], macc[MAXA];
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    sig[a] = a < na ? st.sigma[sb + a] : T(0);
    racc[a] = T(0);
    macc[a] = T(0);
  }
  T r = T(0), m = T(0);  // P64: column tid's running sums (tid < na)
  int32_t ps, ir;
  member_idx(g, m0 + tid, m1, mr, ps, ir);
  for (int32_t k0 = m0; k0 < m1; k0 += kThreads) {
    int32_t qs, jr;  // the next chunk's indices
    member_idx(g, k0 + kThreads + tid, m1, mr, qs, jr);
    T d[MAXA], mm[MAXA];
    member_data<T, MAXA, false>(g, st, k0 + tid, m0, m1, vb, na, p2, sig, ps, ir, d, mm);
    ps = qs;
    ir = jr;
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int a = 0; a < MAXA; ++a) {
        s_d[tid * MAXA + a] = d[a];
        s_m[tid * MAXA + a] = mm[a];
      }
      __syncthreads();
      if (tid < na) {
        const int cnt = (m1 - k0) < kThreads ? (m1 - k0) : kThreads;
        for (int j = 0; j < cnt; ++j) {
          r = r + s_d[j * MAXA + tid];
          m = m + s_m[j * MAXA + tid];
        }
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int a = 0; a < MAXA; ++a) {
        racc[a] += d[a];
        macc[a] += mm[a];
      }
    }
  }
  if (!(upd & (p2 ? 2 : 1))) return;  // alternating updates: values only (uniform over the block)
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      s_d[tid * MAXA + a] = racc[a];
      s_m[tid * MAXA + a] = macc[a];
    }
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
      if (tid < off) {
#pragma unroll
        for (int a = 0; a < MAXA; ++a) {
          s_d[tid * MAXA + a] += s_d[(tid + off) * MAXA + a];
          s_m[tid * MAXA + a] += s_m[(tid + off) * MAXA + a];
        }
      }
      __syncthreads();
    }
    if (tid < na) {
      r = s_d[tid];
      m = s_m[tid];
    }
  }
  // thread a updates slot a (slot_update), then sigma^{t+1} = RM with the
  // positive parts summed in action order
  double pos = 0.0;
  if (tid < na) {
    pos = slot_update(st.R, st.avg, sb + tid, (double)r, (double)m, wt, rule);
    s_pos[tid] = pos;
  }
  __syncthreads();
  if (tid < na) {
    if constexpr (sizeof(T) == 8) {
      double tot = 0.0;
      for (int a = 0; a < na; ++a) tot += s_pos[a];
      st.sigma[sb + tid] = tot > 0.0 ? pos / tot : 1.0 / (double)na;
    } else {
      float tot = 0.f;
      for (int a = 0; a < na; ++a) tot += (float)s_pos[a];
      st.sigma[sb + tid] = tot > 0.f ? (float)pos / tot : 1.f / (float)na;
    }
  }
  __syncthreads();  // shared arrays are reused by the block's next set
}

// Grid: nb_chance blocks over narrow chance nodes, then one block per wide
// chunk, then the information-set groups (LANES == kThreads: one set per
// block).
template <typename T, int MAXA, int LANES>
__global__ void __launch_bounds__(kThreads, MAXA <= 4 ? 4 : (MAXA <= 8 ? 3 : 1)) bwd_level_kernel(GameView g, StateView<T> st, LevelWork w,
                                                            int nb_chance, int rule, int upd, int bump_t) {
  pdl_enter();
  const int nb_wide = w.wc1 - w.wc0;
  if ((int)blockIdx.x < nb_chance) {
    const int32_t stride = nb_chance * blockDim.x;
    for (int32_t i = w.ch0 + blockIdx.x * blockDim.x + threadIdx.x; i < w.ch1; i += stride)
      bwd_chance<T, false>(g, st.v, i);
  } else if ((int)blockIdx.x < nb_chance + nb_wide) {
    bwd_wide_chunk<T, false>(g, w, st.v, w.wc0 + (int32_t)blockIdx.x - nb_chance);
  } else if constexpr (LANES == kThreads) {
    const int first = nb_chance + nb_wide;
    const double wt = avg_weight(*st.t + 1, rule);
    for (int32_t I = w.is0 + ((int)blockIdx.x - first); I < w.is1; I += (int)gridDim.x - first)
      bwd_set_block<T, MAXA>(g, st, I, I >= w.is2, wt, rule, upd);
  } else {
    constexpr int GPB = kThreads / LANES;
    const int first = nb_chance + nb_wide;
    const int gid = ((int)blockIdx.x - first) * GPB + (int)threadIdx.x / LANES;
    const int ngroups = ((int)gridDim.x - first) * GPB;
    const int lane = threadIdx.x % LANES;
    const unsigned mask = group_mask<LANES>();
    const double wt = avg_weight(*st.t + 1, rule);
    for (int32_t I = w.is0 + gid; I < w.is1; I += ngroups)
      bwd_set<T, MAXA, LANES, false>(g, st, I, I >= w.is2, lane, mask, wt, rule, upd);
  }
  if (bump_t) {  // depth 0 holds only the root: no other block reads t here
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) *st.t += 1;
  }
}

static __global__ void bump_t_kernel(long long *t, long long n) { *t += n; }

// ------------------------------------------------------- persistent form
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct Barrier {
  unsigned *count;     // arrivals at the current barrier
  unsigned *gen;       // generation, bumped by the last arrival
  int *err;            // set to 1 when a wait gives up
  long long spin_limit;
  unsigned expected;   // arrivals that complete a barrier (gridDim.x normally)
};

// Grid-wide barrier with a bounded wait: returns false (and sets *err) when
// the spin budget runs out, or when another block has reported an error.
__device__ __forceinline__ bool grid_sync(const Barrier &b) {
  __shared__ int s_ok;
  __syncthreads();
  if (gridDim.x == 1 && b.expected == 1) return true;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned g0 = ld_acquire_gpu(b.gen);
    const unsigned arrived = atomicAdd(b.count, 1u) + 1u;
    int ok = 1;
    if (arrived == b.expected) {
      atomicExch(b.count, 0u);
      __threadfence();
      st_release_gpu(b.gen, g0 + 1u);
    } else {
      long long spins = 0;
      while (ld_acquire_gpu(b.gen) == g0) {
        if (++spins > b.spin_limit) {
          atomicExch(b.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (ok && *(volatile int *)b.err != 0) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T> struct PersistArgs {
  GameView g;
  StateView<T> st;
  const LevelWork *lw;
  int D;
  int rule;
  int order;  // 0 simultaneous, 1 alternating (two half-iterations)
  long long n_iter;
  Barrier bar;
};

// All n iterations in one launch; depth levels separated by grid barriers
// (2D barriers per iteration, 4D under alternating updates). The grid is
// co-resident (cooperative launch).
template <typename T, int MAXA, int LANES>
__global__ void __launch_bounds__(kThreads) persistent_kernel(PersistArgs<T> a) {
  const long long t0 = __ldcg(a.st.t);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int gid = tid / LANES, ngroups = nthr / LANES, lane = tid % LANES;
  const unsigned mask = group_mask<LANES>();
  const int halves = a.order ? 2 : 1;  // alternating: player 1's half, then player 2's
  for (long long it = 0; it < a.n_iter; ++it) {
    const double wt = avg_weight(t0 + it + 1, a.rule);
    for (int hf = 0; hf < halves; ++hf) {
      const int upd = a.order ? (1 << hf) : 3;
      for (int d = 0; d < a.D; ++d) {
        const LevelWork w = a.lw[d];
        if (a.g.int_edge) {  // member order: depth d + 1 pulls
          if (d + 1 < a.D) {
            const int32_t qe = a.lw[d + 1].ie;
            for (int32_t q = a.lw[d + 1].ib + tid; q < qe; q += kPull * nthr)
              fwd_pull<T, true>(a.g, a.st.sigma, a.st.reach, q, nthr, qe);
          }
        } else {
          for (int32_t qw = w.ib + (tid & ~31); qw < w.ie; qw += 4 * nthr) {
            if (w.fan) fwd_int4<T, true, true>(a.g, a.st.sigma, a.st.reach, qw + (tid & 31), nthr, w.ie);
            else fwd_int4<T, true, false>(a.g, a.st.sigma, a.st.reach, qw + (tid & 31), nthr, w.ie);
          }
          for (int32_t q = w.wc0 + blockIdx.x; q < w.wc1; q += gridDim.x) fwd_wide_chunk<T, true>(a.g, w, a.st.reach, q);
        }
        if (!grid_sync(a.bar)) return;
      }
      for (int d = a.D - 1; d >= 0; --d) {
        const LevelWork w = a.lw[d];
        if (d > 0) {  // a chance root's value has no reader in an iteration
          for (int32_t i = w.ch0 + tid; i < w.ch1; i += nthr) bwd_chance<T, true>(a.g, a.st.v, i);
          for (int32_t q = w.wc0 + blockIdx.x; q < w.wc1; q += gridDim.x) bwd_wide_chunk<T, true>(a.g, w, a.st.v, q);
        }
        for (int32_t I = w.is0 + gid; I < w.is1; I += ngroups)
          bwd_set<T, MAXA, LANES, true>(a.g, a.st, I, I >= w.is2, lane, mask, wt, a.rule, upd);
        if (!grid_sync(a.bar)) return;
      }
    }
  }
  if (tid == 0) *a.st.t = t0 + a.n_iter;
}

// ---------------------------------------------------------- state set-up
template <typename T>
__global__ void init_state_kernel(const int32_t *iset_slot, int32_t n_sets, T *sigma, double *R, double *avg,
                                  int32_t A, long long *t, vec2_t<T> *reach, double2 *reach2) {
  const int32_t stride = gridDim.x * blockDim.x;
  const int32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int32_t q = tid; q < A; q += stride) { R[q] = 0.0; avg[q] = 0.0; }
  for (int32_t I = tid; I < n_sets; I += stride) {
    const int32_t sb = iset_slot[I], na = iset_slot[I + 1] - sb;
    for (int32_t a = 0; a < na; ++a) sigma[sb + a] = (T)(1.0 / (double)na);  // RM of zero regret
  }
  if (tid == 0) {
    *t = 0;
    vec2_t<T> one;
    one.x = T(1); one.y = T(1);
    reach[0] = one;  // root reach of both lanes (never overwritten)
    reach2[0] = make_double2(1.0, 1.0);
  }
}

// Every value slot from the template in slot order: terminals get
// pi_c(z) u(z) (eq. (template)), internal nodes 0 (overwritten by every
// backward pass before their parents read them).
template <typename T>
__global__ void init_values_kernel(const double *tmpl_vs, int32_t N, T *v, double2 *vb, double *vavg) {
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < N; h += stride) {
    const double x = tmpl_vs[h];
    v[h] = (T)x;
    vb[h] = make_double2(x, x);
    vavg[h] = x;
  }
}

// sigma from R by regret matching (used after a state upload)
template <typename T>
__global__ void rm_kernel(const int32_t *iset_slot, int32_t n_sets, const double *R, T *sigma) {
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < n_sets; I += stride) {
    const int32_t sb = iset_slot[I], na = iset_slot[I + 1] - sb;
    double tot = 0.0;
    for (int32_t a = 0; a < na; ++a) tot += R[sb + a] > 0.0 ? R[sb + a] : 0.0;
    for (int32_t a = 0; a < na; ++a) {
      const double p = R[sb + a] > 0.0 ? R[sb + a] : 0.0;
      sigma[sb + a] = (T)(tot > 0.0 ? p / tot : 1.0 / (double)na);
    }
  }
}

// ------------------------------------------------------------- read-out
static __global__ void avg_normalize_kernel(const int32_t *iset_slot, int32_t n_sets, const double *avg, double *out) {
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < n_sets; I += stride) {
    const int32_t sb = iset_slot[I], na = iset_slot[I + 1] - sb;
    double tot = 0.0;
    for (int32_t a = 0; a < na; ++a) tot += avg[sb + a];
    for (int32_t a = 0; a < na; ++a) out[sb + a] = tot > 0.0 ? avg[sb + a] / tot : 1.0 / (double)na;
  }
}

template <typename T>
__global__ void to_double_kernel(const T *in, double *out, int32_t n) {
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) out[q] = (double)in[q];
}

// out[spec_slot_of[q]] = in[q]: compiled slot order -> spec slot order
static __global__ void permute_kernel(const int32_t *spec_slot_of, const double *in, double *out, int32_t A) {
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < A; q += stride) out[spec_slot_of[q]] = in[q];
}

// ------------------------------------------------ exact best response (FP64)
// Lane x of vb: player 1 best-responds (maximises), player 2 plays the
// average. Lane y: player 2 best-responds (minimises player 1's payoff),
// player 1 plays the average. vavg: both play the average. All values are
// chance-weighted (eq. (template)), so the counterfactual weight of a member
// is the opponent's reach under the average strategy alone.
// Wide chance node, best-response values: chunk partials of (x, y, avg),
// finished in chunk order by the last block (as bwd_wide_chunk).
__device__ __forceinline__ void br_wide_chunk(const GameView &g, const LevelWork &w, double2 *vb, double *vavg,
                                              int32_t q) {
  const int32_t wi = wide_of_chunk(g, w, q);
  const int32_t h = __ldg(g.wide_vs + wi);
  const int32_t cb = __ldg(g.wide_vb + wi), ce = cb + __ldg(g.wide_nch + wi);
  const int32_t q0 = __ldg(g.wide_chunk + wi), nq = __ldg(g.wide_chunk + wi + 1) - q0;
  const int32_t c0 = cb + (q - q0) * kWideChunkK, c1 = min(ce, c0 + kWideChunkK);
  double sx = 0.0, sy = 0.0, sa = 0.0;
  for (int32_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const double2 x = vb[c];
    sx += x.x; sy += x.y; sa += vavg[c];
  }
  sx = block_sum(sx);
  sy = block_sum(sy);
  sa = block_sum(sa);
  __shared__ unsigned s_ticket;
  if (threadIdx.x == 0) {
    g.wide_part[3 * q] = sx; g.wide_part[3 * q + 1] = sy; g.wide_part[3 * q + 2] = sa;
    __threadfence();
    s_ticket = atomicAdd(g.wide_cnt + wi, 1u);
  }
  __syncthreads();
  if (s_ticket == (unsigned)(nq - 1)) {  // the last chunk's block adds the partials (fixed shape)
    __threadfence();
    double tx = 0.0, ty = 0.0, ta = 0.0;
    for (int32_t k = threadIdx.x; k < nq; k += blockDim.x) {
      tx += __ldcg(g.wide_part + 3 * (q0 + k));
      ty += __ldcg(g.wide_part + 3 * (q0 + k) + 1);
      ta += __ldcg(g.wide_part + 3 * (q0 + k) + 2);
    }
    tx = block_sum(tx);
    ty = block_sum(ty);
    ta = block_sum(ta);
    if (threadIdx.x == 0) {
      vb[h] = make_double2(tx, ty);
      vavg[h] = ta;
      g.wide_cnt[wi] = 0u;
    }
  }
}

template <int MAXA, int LANES>
__global__ void __launch_bounds__(kThreads) br_level_kernel(GameView g, const double2 *reach2, const double *sbs,
                                                           double2 *vb, double *vavg, LevelWork w, int nb_chance) {
  const int nb_wide = w.wc1 - w.wc0;
  if ((int)blockIdx.x >= nb_chance && (int)blockIdx.x < nb_chance + nb_wide) {
    br_wide_chunk(g, w, vb, vavg, w.wc0 + (int32_t)blockIdx.x - nb_chance);
    return;
  }
  if ((int)blockIdx.x < nb_chance) {
    const int32_t stride = nb_chance * blockDim.x;
    for (int32_t i = w.ch0 + blockIdx.x * blockDim.x + threadIdx.x; i < w.ch1; i += stride) {
      const int32_t h = __ldg(g.ch_vs + i);
      const int32_t cb = __ldg(g.ch_vb + i), ce = cb + __ldg(g.ch_nch + i);
      double sx = 0.0, sy = 0.0, sa = 0.0;
      for (int32_t c = cb; c < ce; ++c) { const double2 x = vb[c]; sx += x.x; sy += x.y; sa += vavg[c]; }
      vb[h] = make_double2(sx, sy);
      vavg[h] = sa;
    }
    return;
  }
  constexpr int GPB = kThreads / LANES;
  const int first = nb_chance + nb_wide;
  const int gid = ((int)blockIdx.x - first) * GPB + (int)threadIdx.x / LANES;
  const int ngroups = ((int)gridDim.x - first) * GPB;
  const int lane = threadIdx.x % LANES;
  const unsigned mask = group_mask<LANES>();
  for (int32_t I = w.is0 + gid; I < w.is1; I += ngroups) {
    const int p = I >= w.is2 ? 1 : 0;
    const int32_t sb = __ldg(g.iset_slot + I), na = __ldg(g.iset_slot + I + 1) - sb;
    const int32_t m0 = __ldg(g.iset_mem + I), m1 = __ldg(g.iset_mem + I + 1);
    const MemberRanks mr = member_ranks(g, I, m0);
    const int32_t vb0 = __ldg(g.iset_vb + I);
    double sg[MAXA], Q[MAXA];
#pragma unroll
    for (int a = 0; a < MAXA; ++a) { sg[a] = a < na ? sbs[sb + a] : 0.0; Q[a] = 0.0; }
    for (int32_t k0 = m0; k0 < m1; k0 += LANES) {
      const int32_t k = k0 + lane;
      double q[MAXA];
#pragma unroll
      for (int a = 0; a < MAXA; ++a) q[a] = 0.0;
      if (k < m1) {
        const int32_t h = __ldg(g.mem_vs + k);
        const int32_t cb = vb0 + (k - m0), M = m1 - m0;
        const double2 r = reach2[member_rank(g, k, mr)];
        const double po = p ? r.x : r.y;
        double oth = 0.0, va = 0.0;
#pragma unroll
        for (int a = 0; a < MAXA; ++a) {
          if (a < na) {
            const double2 x = vb[cb + a * M];
            q[a] = po * (p ? x.y : x.x);
            oth += sg[a] * (p ? x.x : x.y);
            va += sg[a] * vavg[cb + a * M];
          }
        }
        reinterpret_cast<double *>(vb + h)[1 - p] = oth;
        vavg[h] = va;
      }
      const int cnt = (m1 - k0) < LANES ? (m1 - k0) : LANES;
      for (int j = 0; j < cnt; ++j) {
#pragma unroll
        for (int a = 0; a < MAXA; ++a)
          if (a < na) Q[a] += __shfl_sync(mask, q[a], j, LANES);
      }
    }
    int best = 0;
    for (int a = 1; a < na; ++a)
      if (p == 0 ? Q[a] > Q[best] : Q[a] < Q[best]) best = a;
    // every lane computed the same Q (the ordered sums are broadcast), so
    // best agrees across the group without another shuffle
    for (int32_t k = m0 + lane; k < m1; k += LANES) {
      const int32_t h = __ldg(g.mem_vs + k);
      const int32_t cb = vb0 + (k - m0) + best * (m1 - m0);
      reinterpret_cast<double *>(vb + h)[p] = reinterpret_cast<const double *>(vb + cb)[p];
    }
  }
}

}  // namespace cfr
