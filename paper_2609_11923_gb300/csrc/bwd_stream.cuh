// bwd_stream.cuh — the FP32 backward pass of one depth with its inputs
// streamed into shared memory by the bulk-copy (TMA) engine.
//
// Same arithmetic as bwd_set (eqs. (opbwd), (instregret), (regret), (rm), the
// CFR+ clamp; Algorithm 1), different data movement. In member order the
// information sets of a depth are a contiguous range and so is everything a
// run of consecutive sets reads: their members' reach (one run, tiles
// interleaved inside it), their members' children's values (one run of value
// slots), their members' own value slots, their slots' strategy, regret and
// average, and their set descriptors. The host cuts each depth's sets into
// chunks of whole groups (a tile of four sets, or one untiled set) whose
// staged bytes fit one pipeline stage. Every CTA walks the chunks c =
// blockIdx, blockIdx + grid, ... through a ring of kStreamStages stages: one
// thread issues the chunk's seven cp.async.bulk copies into a stage and the
// stage's mbarrier counts their bytes; all threads wait on the mbarrier
// (bounded), compute the chunk from shared memory, and the stage is refilled
// with the chunk kStreamStages ahead. The loads in flight cost no registers,
// so the memory pipe stays full at a low warp count; the one scattered access
// left is each member's value write into its parent set's block.
//
// Work inside a chunk: the CTA takes one group at a time with all its
// threads; thread t serves set j = t % G of the group (G = 4 for a tile,
// 1 otherwise) and members q = t / G, t / G + 256 / G, ... of that set, so a
// warp reads a tile's reach as one contiguous run. Per-thread FP32 partial
// sums are finished by a fixed-shape butterfly within the warp and a sum over
// the warps in warp order (deterministic run to run), then warp 0 updates the
// group's slots (one lane per slot) and writes sigma^{t+1}.
#pragma once
#include "kernels.cuh"

namespace cfr {

constexpr int kStreamLanes = 512;                 // lanes_per_set code of this form
constexpr int kStreamStages = 2;                  // pipeline depth
constexpr int kStreamStageBytes = 48 * 1024;      // bytes one chunk may stage
constexpr int kStreamWarps = kThreads / 32;

// Per information set (member order), 32 bytes, read by the streaming form.
struct SetInfo {
  int32_t sb, na;        // first slot, actions
  int32_t m0, nm;        // first member, member count
  int32_t vb;            // first value slot of the block of its members' children
  int32_t rank0, rstep;  // reach rank of member 0 and the stride of its members' ranks
  int32_t flags;         // bits 0-2: G (sets in the group it starts: 1 or 4; 0 inside a tile); bit 8: player 2
};

// One chunk of consecutive sets [I0, I1) and the element ranges it stages,
// widened to 16-byte boundaries: reach ranks [ra, ra + nra) (even), value
// slots [va, va + nva), members [ka, ka + nka), slots [sa, sa + nsa)
// (multiples of 4).
struct StreamChunk {
  int32_t I0, I1;
  int32_t ra, nra;
  int32_t va, nva;
  int32_t ka, nka;
  int32_t sa, nsa;
  int32_t pad[6];
};

static_assert(sizeof(SetInfo) == 32, "SetInfo is staged in 32-byte records");
static_assert(sizeof(StreamChunk) == 64, "StreamChunk is 64 bytes");

// Byte offsets of the staged arrays inside one stage.
struct StreamLayout {
  uint32_t reach, val, mem, info, sig, R, avg, total;
};

__host__ __device__ inline StreamLayout stream_layout(const StreamChunk &c) {
  StreamLayout L;
  L.reach = 0;
  L.val = L.reach + 8u * (uint32_t)c.nra;
  L.mem = L.val + 4u * (uint32_t)c.nva;
  L.info = L.mem + 4u * (uint32_t)c.nka;
  L.sig = L.info + (uint32_t)sizeof(SetInfo) * (uint32_t)(c.I1 - c.I0);
  L.R = L.sig + 4u * (uint32_t)c.nsa;
  L.avg = L.R + 8u * (uint32_t)c.nsa;
  L.total = L.avg + 8u * (uint32_t)c.nsa;
  return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completing `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Bounded wait for the phase of the given parity: false when it gave up
// (about a second of polling).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 26); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 4000000000ll) break;
  }
  return false;
}

// Issues the copies of chunk d into a stage (one thread). Returns false (and
// issues nothing) if the chunk does not fit the stage.
__device__ __forceinline__ bool stream_issue(const StreamChunk &d, unsigned char *stage, uint32_t bar,
                                             const float2 *reach, const float *v, const int32_t *mem_vs,
                                             const SetInfo *info, const float *sigma, const double *R,
                                             const double *avg) {
  const StreamLayout L = stream_layout(d);
  if (L.total > (uint32_t)kStreamStageBytes || d.nra <= 0 || d.nva <= 0 || d.nka <= 0 || d.I1 <= d.I0 || d.nsa <= 0)
    return false;
  const uint32_t s = smem_u32(stage);
  mbar_expect_tx(bar, L.total);  // the seven sizes below add up to L.total
  bulk_g2s(s + L.reach, reach + d.ra, L.val - L.reach, bar);
  bulk_g2s(s + L.val, v + d.va, L.mem - L.val, bar);
  bulk_g2s(s + L.mem, mem_vs + d.ka, L.info - L.mem, bar);
  bulk_g2s(s + L.info, info + d.I0, L.sig - L.info, bar);
  bulk_g2s(s + L.sig, sigma + d.sa, L.R - L.sig, bar);
  bulk_g2s(s + L.R, R + d.sa, L.avg - L.R, bar);
  bulk_g2s(s + L.avg, avg + d.sa, L.total - L.avg, bar);
  return true;
}

// One group of sets (G = 1 or 4) of a staged chunk, all threads.
template <int MAXA>
__device__ __forceinline__ void stream_group(const StreamChunk &d, const StreamLayout &L, const unsigned char *stage,
                                             int32_t I, float *v, float *sigma, double *Rg, double *avgg, double wt,
                                             int rule, int upd, float (*red)[4][2 * MAXA]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SetInfo *sinfo = reinterpret_cast<const SetInfo *>(stage + L.info);
  const int G = sinfo[I - d.I0].flags & 7;  // 1 or 4
  const int gs = G == 4 ? 2 : 0;
  const int j = tid & (G - 1);
  const int LPS = kThreads >> gs;
  const SetInfo si = sinfo[I + j - d.I0];
  const bool p2 = (si.flags >> 8) & 1;
  const float2 *sr = reinterpret_cast<const float2 *>(stage + L.reach);
  const float *sv = reinterpret_cast<const float *>(stage + L.val);
  const int32_t *sm = reinterpret_cast<const int32_t *>(stage + L.mem);
  const float *ss = reinterpret_cast<const float *>(stage + L.sig);
  float sig[MAXA], racc[MAXA], macc[MAXA];
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    sig[a] = a < si.na ? ss[si.sb - d.sa + a] : 0.f;
    racc[a] = 0.f;
    macc[a] = 0.f;
  }
  const int32_t rb = si.rank0 - d.ra, kb = si.m0 - d.ka, cbase = si.vb - d.va;
  for (int32_t q = tid >> gs; q < si.nm; q += LPS) {
    const float2 r = sr[rb + q * si.rstep];
    const int32_t h = sm[kb + q];
    const int32_t cb = cbase + q * si.na;
    float vc[MAXA];
    float vh = 0.f;
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      if (a < si.na) {
        vc[a] = sv[cb + a];
        vh = vh + sig[a] * vc[a];
      }
    }
    v[h] = vh;
    const float po = p2 ? r.x : r.y;  // opponent's reach (chance is inside v)
    const float pw = p2 ? r.y : r.x;  // own reach
    const float f = (p2 ? -1.f : 1.f) * po;
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      if (a < si.na) {
        racc[a] += f * (vc[a] - vh);
        macc[a] += pw * sig[a];
      }
    }
  }
  // butterfly over the lanes of the warp that serve the same set
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    for (int off = G; off < 32; off <<= 1) {
      racc[a] += __shfl_xor_sync(0xffffffffu, racc[a], off);
      macc[a] += __shfl_xor_sync(0xffffffffu, macc[a], off);
    }
  }
  if (lane < G) {
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      red[warp][lane][a] = racc[a];
      red[warp][lane][MAXA + a] = macc[a];
    }
  }
  __syncthreads();
  if (warp != 0) return;
  // warp 0: lane = a * G + jj updates slot a of set jj of the group
  const int jj = lane & (G - 1), a = lane >> gs;
  const SetInfo sj = sinfo[I + jj - d.I0];
  const bool q2 = (sj.flags >> 8) & 1;
  const bool live = a < MAXA && a < sj.na;
  float pf = 0.f;
  if (live && (upd & (q2 ? 2 : 1))) {
    float r = 0.f, m = 0.f;
    for (int w = 0; w < kStreamWarps; ++w) {  // warps in order
      r += red[w][jj][a];
      m += red[w][jj][MAXA + a];
    }
    const int32_t qs = sj.sb + a;
    const double *sR = reinterpret_cast<const double *>(stage + L.R);
    const double *sA = reinterpret_cast<const double *>(stage + L.avg);
    double Rn = sR[qs - d.sa] + (double)r;
    if (rule != kRuleCfr) Rn = Rn > 0.0 ? Rn : 0.0;
    Rg[qs] = Rn;
    avgg[qs] = sA[qs - d.sa] + wt * (double)m;
    const double x = rule == kRulePcfrPlus ? Rn + (double)r : Rn;
    pf = (float)(x > 0.0 ? x : 0.0);
  }
  float tot = 0.f;  // positive parts in action order
  for (int b = 0; b < MAXA; ++b) {
    const float x = __shfl_sync(0xffffffffu, pf, (b * G + jj) & 31);
    if (b < sj.na) tot += x;
  }
  if (live && (upd & (q2 ? 2 : 1))) sigma[sj.sb + a] = tot > 0.f ? pf / tot : 1.f / (float)sj.na;
}

// Grid: nb_chance blocks over narrow chance nodes, then one block per wide
// chunk, then the streaming CTAs over chunks [c0, c1) of this depth.
template <int MAXA>
__global__ void __launch_bounds__(kThreads, 2)
    bwd_stream_kernel(GameView g, StateView<float> st, LevelWork w, int nb_chance, const SetInfo *info,
                      const StreamChunk *chunks, int32_t c0, int32_t c1, int rule, int upd, int *err) {
  extern __shared__ __align__(128) unsigned char s_stage[];
  __shared__ __align__(8) uint64_t s_bar[kStreamStages];
  __shared__ StreamChunk s_desc[kStreamStages];
  __shared__ float s_red[2][kStreamWarps][4][2 * MAXA];
  __shared__ int s_fail;
  __shared__ int s_issued[kStreamStages];  // a stage has copies in flight or landed, not yet consumed
  const int nb_wide = w.wc1 - w.wc0;
  if ((int)blockIdx.x < nb_chance) {
    const int32_t stride = nb_chance * blockDim.x;
    for (int32_t i = w.ch0 + blockIdx.x * blockDim.x + threadIdx.x; i < w.ch1; i += stride)
      bwd_chance<float, false>(g, st.v, i);
    return;
  }
  if ((int)blockIdx.x < nb_chance + nb_wide) {
    bwd_wide_chunk<float, false>(g, w, st.v, w.wc0 + (int32_t)blockIdx.x - nb_chance);
    return;
  }
  const int32_t b = (int32_t)blockIdx.x - nb_chance - nb_wide;
  const int32_t nb = (int32_t)gridDim.x - nb_chance - nb_wide;
  const int tid = threadIdx.x;
  const double wt = avg_weight(*st.t + 1, rule);
  if ((smem_u32(s_stage) & 15u) != 0u) {  // bulk copies need 16-byte aligned destinations
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < kStreamStages; ++s) {
      mbar_init(smem_u32(&s_bar[s]), 1);
      s_issued[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  // prologue: the first kStreamStages chunks of this CTA
  if (tid == 0) {
    for (int s = 0; s < kStreamStages; ++s) {
      const int32_t c = c0 + b + s * nb;
      if (c >= c1) break;
      s_desc[s] = chunks[c];
      if (!stream_issue(s_desc[s], s_stage + s * kStreamStageBytes, smem_u32(&s_bar[s]), st.reach, st.v, g.mem_vs,
                        info, st.sigma, st.R, st.avg)) {
        s_fail = 1;
        atomicExch(err, 1);
        break;
      }
      s_issued[s] = 1;
    }
  }
  __syncthreads();
  if (s_fail) return;
  int par = 0;
  for (int32_t i = 0;; ++i) {
    const int32_t c = c0 + b + i * nb;
    if (c >= c1) break;
    const int s = i % kStreamStages;
    const uint32_t parity = (uint32_t)((i / kStreamStages) & 1);
    // the descriptor of the chunk this stage takes next (its load overlaps the compute)
    const int32_t cn = c + kStreamStages * nb;
    StreamChunk nd;
    if (tid == 0 && cn < c1) nd = chunks[cn];
    const bool have = s_issued[s] != 0;
    if (have && !mbar_wait(smem_u32(&s_bar[s]), parity)) atomicExch(&s_fail, 1);
    __syncthreads();
    if (s_fail || !have) {
      // give up: let the copies still in flight into the other stages land
      // (bounded), then leave
      if (tid == 0) {
        atomicExch(err, 1);
        for (int k = 1; k < kStreamStages; ++k)
          if (s_issued[(s + k) % kStreamStages])
            mbar_wait(smem_u32(&s_bar[(s + k) % kStreamStages]), (uint32_t)(((i + k) / kStreamStages) & 1));
      }
      return;
    }
    const StreamChunk d = s_desc[s];
    const StreamLayout L = stream_layout(d);
    const unsigned char *stage = s_stage + s * kStreamStageBytes;
    const SetInfo *sinfo = reinterpret_cast<const SetInfo *>(stage + L.info);
    for (int32_t I = d.I0; I < d.I1;) {
      const int G = sinfo[I - d.I0].flags & 7;
      stream_group<MAXA>(d, L, stage, I, st.v, st.sigma, st.R, st.avg, wt, rule, upd, s_red[par]);
      par ^= 1;
      I += G;
    }
    __syncthreads();  // every thread is done with the stage
    if (tid == 0) {
      s_issued[s] = 0;
      if (cn < c1) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_desc[s] = nd;
        if (stream_issue(nd, s_stage + s * kStreamStageBytes, smem_u32(&s_bar[s]), st.reach, st.v, g.mem_vs, info,
                         st.sigma, st.R, st.avg))
          s_issued[s] = 1;
        else
          atomicExch(err, 1);  // the next wait on this stage sees it unissued and leaves
      }
    }
  }
}

}  // namespace cfr
