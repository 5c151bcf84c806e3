// batch.cuh — many independent solves in one launch (batched serving).
//
// One CTA owns one instance for the whole call: it runs that instance's n
// CFR+ iterations with __syncthreads() between depth levels (no grid
// barrier, no cross-CTA traffic), so a batch of hundreds of uneven
// subgames is one launch whose CTAs the hardware schedules as SMs free up.
// Large instances instead get a thread-block cluster of several CTAs (the
// clustered instances of the kernel, launched with a cluster dimension):
// the cluster's CTAs share each depth's work and meet at the hardware
// cluster barrier (barrier.cluster, release/acquire) between depths, and
// read the state arrays through L2 because their L1s are not coherent.
// Each instance's arithmetic depends only on its own arrays and on the
// launch shape (THREADS, LANES, cluster size): a solve gives bitwise the
// same result alone and inside any mix run with the same shape. The
// per-level device functions are the ones of kernels.cuh; wide chance nodes
// are summed by one CTA in a fixed order.
#pragma once
#include "kernels.cuh"

namespace cfr {

// Everything a CTA needs about one bound instance (device pointers into the
// instance's own arena).
struct InstDesc {
  GameView g;
  void *reach;
  void *v;
  void *sigma;
  double *R;
  double *avg;
  long long *t;
  const LevelWork *lw;
  double2 *reach2;
  double2 *vb;
  double *vavg;
  double *sbs;
  double *out;      // exploitability result slot (batch_br_kernel)
  long long n_iter; // iterations this call runs for the instance
  int32_t D;
  int32_t rule;
  int32_t n_sets;
  int32_t root_vs;  // the root's value slot (N - 1)
  int32_t order;    // 0 simultaneous, 1 alternating updates
  int32_t pad;
};

template <int THREADS>
__device__ __forceinline__ double cta_sum(double x, double *sm) {
  __syncthreads();
  sm[threadIdx.x] = x;
  __syncthreads();
#pragma unroll
  for (int s = THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

// Cluster geometry (1 and 0 outside a cluster launch) and the barrier
// between depths: the CTA barrier, or the cluster barrier whose release /
// acquire makes each CTA's global writes visible to the others.
__device__ __forceinline__ unsigned cluster_ncta() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
template <bool CLUSTERED>
__device__ __forceinline__ void level_sync() {
  if constexpr (CLUSTERED)
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  else
    __syncthreads();
}

// Wide chance node: its internal children copy its reach (thread ct of NT).
template <typename T, bool PERSIST>
__device__ __forceinline__ void cta_fwd_wide(const GameView &g, vec2_t<T> *reach, int32_t wi, int ct, int NT) {
  const int32_t ir = __ldg(g.wide_irank + wi);
  const int32_t off = __ldg(g.int_cirank + ir);
  const int32_t nch = __ldg(g.big_irank + off);
  const vec2_t<T> r = ldm<PERSIST>(reach + ir);
  for (int32_t j = ct; j < nch; j += NT) {
    const int32_t c = __ldg(g.big_irank + off + 1 + j);
    if (c >= 0) reach[c] = r;
  }
}

// Wide chance node wi inside one CTA: value = sum of the children's values.
// P64 sums left to right (thread 0); P32 uses the fixed-shape CTA tree.
template <typename T, int THREADS, bool PERSIST>
__device__ __forceinline__ void cta_bwd_wide(const GameView &g, T *v, int32_t wi, double *sm) {
  const int32_t h = __ldg(g.wide_vs + wi);
  const int32_t cb = __ldg(g.wide_vb + wi), ce = cb + __ldg(g.wide_nch + wi);
  if constexpr (sizeof(T) == 8) {
    const double s = ordered_sum<THREADS, PERSIST>(v, cb, ce);
    if (threadIdx.x == 0) v[h] = s;
  } else {
    double x = 0.0;
    for (int32_t c = cb + threadIdx.x; c < ce; c += THREADS) x += (double)ldm<PERSIST>(v + c);
    x = cta_sum<THREADS>(x, sm);
    if (threadIdx.x == 0) v[h] = (T)x;
  }
}

template <typename T, int MAXA, int LANES, int THREADS, bool CLUSTERED>
__global__ void __launch_bounds__(THREADS) batch_iterate_kernel(const InstDesc *table, int n_inst) {
  __shared__ double sm[THREADS];
  const int ncta = CLUSTERED ? (int)cluster_ncta() : 1;   // CTAs sharing this instance
  const int rank = CLUSTERED ? (int)cluster_rank() : 0;
  const int inst = (int)blockIdx.x / ncta;
  if (inst >= n_inst) return;  // the whole cluster leaves together
  const int ct = rank * THREADS + (int)threadIdx.x, NT = ncta * THREADS;
  const InstDesc in = table[inst];
  StateView<T> st;
  st.reach = (vec2_t<T> *)in.reach;
  st.v = (T *)in.v;
  st.sigma = (T *)in.sigma;
  st.R = in.R;
  st.avg = in.avg;
  st.t = in.t;
  const long long t0 = *in.t;
  const int lane = threadIdx.x % LANES, gid = ct / LANES;
  const int NG = NT / LANES;
  const unsigned mask = group_mask<LANES>();
  const int halves = in.order ? 2 : 1;  // alternating: player 1's half, then player 2's
  for (long long it = 0; it < in.n_iter; ++it) {
    const double wt = avg_weight(t0 + it + 1, in.rule);
    for (int hf = 0; hf < halves; ++hf) {
      const int upd = in.order ? (1 << hf) : 3;
      for (int d = 0; d < in.D; ++d) {
        const LevelWork w = in.lw[d];
        if (in.g.int_edge) {  // member order: depth d + 1 pulls
          if (d + 1 < in.D) {
            const int32_t qe = in.lw[d + 1].ie;
            for (int32_t q = in.lw[d + 1].ib + ct; q < qe; q += kPull * NT)
              fwd_pull<T, CLUSTERED>(in.g, st.sigma, st.reach, q, NT, qe);
          }
        } else {
          for (int32_t qw = w.ib + rank * THREADS + (threadIdx.x & ~31); qw < w.ie; qw += 4 * NT) {
            if (w.fan) fwd_int4<T, CLUSTERED, true>(in.g, st.sigma, st.reach, qw + (threadIdx.x & 31), NT, w.ie);
            else fwd_int4<T, CLUSTERED, false>(in.g, st.sigma, st.reach, qw + (threadIdx.x & 31), NT, w.ie);
          }
          for (int32_t i = w.wd0; i < w.wd1; ++i) cta_fwd_wide<T, CLUSTERED>(in.g, st.reach, i, ct, NT);
        }
        level_sync<CLUSTERED>();
      }
      for (int d = in.D - 1; d >= 0; --d) {
        const LevelWork w = in.lw[d];
        if (d > 0) {  // a chance root's value has no reader in an iteration
          for (int32_t i = w.ch0 + ct; i < w.ch1; i += NT)
            bwd_chance<T, CLUSTERED>(in.g, st.v, i);
          if (rank == 0)
            for (int32_t i = w.wd0; i < w.wd1; ++i) cta_bwd_wide<T, THREADS, CLUSTERED>(in.g, st.v, i, sm);
        }
        // 1024-thread blocks leave 64 registers a thread: lean average terms
        for (int32_t I = w.is0 + gid; I < w.is1; I += NG)
          bwd_set<T, MAXA, LANES, CLUSTERED, (THREADS >= 1024)>(in.g, st, I, I >= w.is2, lane, mask, wt, in.rule, upd);
        level_sync<CLUSTERED>();
      }
    }
  }
  if (ct == 0) *in.t = t0 + in.n_iter;
}

// Exploitability of every instance's average strategy (FP64), one CTA each:
// normalise the average, forward reach under it, then both best responses by
// depth (the same arithmetic as br_level_kernel, with CTA-wide loops).
template <int MAXA, int LANES, int THREADS>
__global__ void __launch_bounds__(THREADS) batch_br_kernel(const InstDesc *table, int n_inst) {
  __shared__ double sm[THREADS];
  const int inst = blockIdx.x;
  if (inst >= n_inst) return;
  const InstDesc in = table[inst];
  const GameView &g = in.g;
  // average strategy, normalised per set
  for (int32_t I = threadIdx.x; I < in.n_sets; I += THREADS) {
    const int32_t sb = __ldg(g.iset_slot + I), na = __ldg(g.iset_slot + I + 1) - sb;
    double tot = 0.0;
    for (int32_t a = 0; a < na; ++a) tot += in.avg[sb + a];
    for (int32_t a = 0; a < na; ++a) in.sbs[sb + a] = tot > 0.0 ? in.avg[sb + a] / tot : 1.0 / (double)na;
  }
  __syncthreads();
  for (int d = 0; d < in.D; ++d) {
    const LevelWork w = in.lw[d];
    if (g.int_edge) {  // member order: depth d + 1 pulls
      if (d + 1 < in.D) {
        const int32_t qe = in.lw[d + 1].ie;
        for (int32_t q = in.lw[d + 1].ib + (int32_t)threadIdx.x; q < qe; q += kPull * THREADS)
          fwd_pull<double, false>(g, in.sbs, in.reach2, q, THREADS, qe);
      }
    } else {
      for (int32_t qw = w.ib + (threadIdx.x & ~31); qw < w.ie; qw += 4 * THREADS) {
        if (w.fan) fwd_int4<double, false, true>(g, in.sbs, in.reach2, qw + (threadIdx.x & 31), THREADS, w.ie);
        else fwd_int4<double, false, false>(g, in.sbs, in.reach2, qw + (threadIdx.x & 31), THREADS, w.ie);
      }
      for (int32_t i = w.wd0; i < w.wd1; ++i) cta_fwd_wide<double, false>(g, in.reach2, i, threadIdx.x, THREADS);
    }
    __syncthreads();
  }
  const int lane = threadIdx.x % LANES, gid = threadIdx.x / LANES;
  constexpr int NG = THREADS / LANES;
  const unsigned mask = group_mask<LANES>();
  for (int d = in.D - 1; d >= 0; --d) {
    const LevelWork w = in.lw[d];
    for (int32_t i = w.ch0 + threadIdx.x; i < w.ch1; i += THREADS) {
      const int32_t h = __ldg(g.ch_vs + i);
      const int32_t cb = __ldg(g.ch_vb + i), ce = cb + __ldg(g.ch_nch + i);
      double sx = 0.0, sy = 0.0, sa = 0.0;
      for (int32_t c = cb; c < ce; ++c) { const double2 x = in.vb[c]; sx += x.x; sy += x.y; sa += in.vavg[c]; }
      in.vb[h] = make_double2(sx, sy);
      in.vavg[h] = sa;
    }
    for (int32_t i = w.wd0; i < w.wd1; ++i) {
      const int32_t h = __ldg(g.wide_vs + i);
      const int32_t cb = __ldg(g.wide_vb + i), ce = cb + __ldg(g.wide_nch + i);
      double sx = 0.0, sy = 0.0, sa = 0.0;
      for (int32_t c = cb + threadIdx.x; c < ce; c += THREADS) { const double2 x = in.vb[c]; sx += x.x; sy += x.y; sa += in.vavg[c]; }
      sx = cta_sum<THREADS>(sx, sm);
      sy = cta_sum<THREADS>(sy, sm);
      sa = cta_sum<THREADS>(sa, sm);
      if (threadIdx.x == 0) { in.vb[h] = make_double2(sx, sy); in.vavg[h] = sa; }
    }
    for (int32_t I = w.is0 + gid; I < w.is1; I += NG) {
      const int p = I >= w.is2 ? 1 : 0;
      const int32_t sb = __ldg(g.iset_slot + I), na = __ldg(g.iset_slot + I + 1) - sb;
      const int32_t m0 = __ldg(g.iset_mem + I), m1 = __ldg(g.iset_mem + I + 1);
      const MemberRanks mr = member_ranks(g, I, m0);
      const int32_t vb0 = __ldg(g.iset_vb + I);
      double sg[MAXA], Q[MAXA];
#pragma unroll
      for (int a = 0; a < MAXA; ++a) { sg[a] = a < na ? in.sbs[sb + a] : 0.0; Q[a] = 0.0; }
      for (int32_t k0 = m0; k0 < m1; k0 += LANES) {
        const int32_t k = k0 + lane;
        double q[MAXA];
#pragma unroll
        for (int a = 0; a < MAXA; ++a) q[a] = 0.0;
        if (k < m1) {
          const int32_t h = __ldg(g.mem_vs + k);
          const int32_t cb = vb0 + (k - m0), M = m1 - m0;
          const double2 r = in.reach2[member_rank(g, k, mr)];
          const double po = p ? r.x : r.y;
          double oth = 0.0, va = 0.0;
#pragma unroll
          for (int a = 0; a < MAXA; ++a) {
            if (a < na) {
              const double2 x = in.vb[cb + a * M];
              q[a] = po * (p ? x.y : x.x);
              oth += sg[a] * (p ? x.x : x.y);
              va += sg[a] * in.vavg[cb + a * M];
            }
          }
          reinterpret_cast<double *>(in.vb + h)[1 - p] = oth;
          in.vavg[h] = va;
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
      for (int32_t k = m0 + lane; k < m1; k += LANES) {
        const int32_t h = __ldg(g.mem_vs + k);
        const int32_t cb = vb0 + (k - m0) + best * (m1 - m0);
        reinterpret_cast<double *>(in.vb + h)[p] = reinterpret_cast<const double *>(in.vb + cb)[p];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double2 root = in.vb[in.root_vs];
    in.out[0] = 0.5 * (root.x - root.y);
    in.out[1] = root.x;
    in.out[2] = root.y;
    in.out[3] = in.vavg[in.root_vs];
  }
}

}  // namespace cfr
