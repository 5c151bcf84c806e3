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
// staged bytes fit one pipeline stage; the depth's narrow chance nodes
// follow as chance chunks (consecutive nodes, whose children are one run of
// value slots, and their entries of the chance arrays), summed in the same
// pipeline. Every CTA walks the chunks c = blockIdx, blockIdx + grid, ...
// through a ring of kStreamStages stages. Its kStreamCompute compute threads
// do the members' (or chance nodes') work; the copy warp issues each chunk's
// cp.async.bulk copies into a stage and a side slot (their mbarriers count
// the bytes), and the update warp runs every group's slot update.
// The loads in flight cost no registers, so the memory pipe stays full at a
// low warp count, and the compute warps never wait for a slot update (they
// hand each group's partial sums over through a double-buffered array and a
// pair of mbarriers); the one scattered access left is each member's value
// write into its parent set's block.
//
// Work inside a chunk: the compute threads take one group at a time: thread
// t serves set j = t % G of the group (G = 4 for a tile, 1 otherwise) and
// members q = t / G, t / G + 256 / G, ... of that set, so a warp reads a
// tile's reach as one contiguous run. Per-thread FP32 partial sums are
// finished by a fixed-shape butterfly within the warp and, in the update
// warp, a sum over the warps in warp order (deterministic run to run); the
// update warp then updates the group's slots (one lane per slot) and writes
// sigma^{t+1}. The form pays where sets are long (hundreds of members).
#pragma once
#include "kernels.cuh"

namespace cfr {

constexpr int kStreamLanes = 512;                 // lanes_per_set code of this form
constexpr int kStreamStages = 2;                  // pipeline depth
constexpr int kStreamStageBytes = 48 * 1024;      // bytes one chunk may stage for the compute threads
constexpr int kStreamSideSlots = 4;               // ring of the update warp's per-chunk data
constexpr int kStreamSideBytes = 2048;            // bytes of one side slot
constexpr int kStreamDynSmem = kStreamStages * kStreamStageBytes + kStreamSideSlots * kStreamSideBytes;
constexpr int kStreamCompute = 256;               // compute threads of a streaming CTA (two CTAs per SM)
constexpr int kStreamWarps = kStreamCompute / 32;
constexpr int kStreamMinMembers = 32;             // mean members per set below which the autotuner does not try it
constexpr int kStreamChanceMax = 4 * kStreamCompute;  // chance nodes per chance chunk at most

// Per information set (member order), 32 bytes, read by the streaming form.
struct SetInfo {
  int32_t sb, na;        // first slot, actions
  int32_t m0, nm;        // first member, member count
  int32_t vb;            // first value slot of the block of its members' children
  int32_t rank0, rstep;  // reach rank of member 0 and the stride of its members' ranks
  int32_t flags;         // bits 0-2: G (sets in the group it starts: 1 or 4; 0 inside a tile); bit 8: player 2
};

// One chunk and the element ranges it stages, widened to 16-byte
// boundaries. A set chunk (kind kChunkSets): consecutive sets [I0, I1),
// reach ranks [ra, ra + nra) (even), value slots [va, va + nva), members
// [ka, ka + nka), slots [sa, sa + nsa) (multiples of 4). A chance chunk
// (kind kChunkChance): consecutive narrow chance nodes [I0, I1) of the
// depth, their children's value slots [va, va + nva) and their entries
// [ka, ka + nka) of the chance arrays (first child slot, child count, own
// value slot); ra = nra = sa = nsa = 0.
constexpr int32_t kChunkSets = 0, kChunkChance = 1;
struct StreamChunk {
  int32_t I0, I1;
  int32_t ra, nra;
  int32_t va, nva;
  int32_t ka, nka;
  int32_t sa, nsa;
  int32_t kind;
  int32_t pad[5];
};

static_assert(sizeof(SetInfo) == 32, "SetInfo is staged in 32-byte records");
static_assert(sizeof(StreamChunk) == 64, "StreamChunk is 64 bytes");

// Byte offsets of the staged arrays: in a stage (what the compute threads
// read) and in a side slot (what the update warp reads for the slot
// updates, so that the stage can be refilled while it still works).
struct StreamLayout {
  uint32_t reach, val, mem, info, sig, total;  // stage
  uint32_t s_info, s_R, s_avg, s_total;        // side slot
};

__host__ __device__ inline StreamLayout stream_layout(const StreamChunk &c) {
  StreamLayout L;
  const uint32_t nset = (uint32_t)sizeof(SetInfo) * (uint32_t)(c.I1 - c.I0);
  L.reach = 0;
  L.val = L.reach + 8u * (uint32_t)c.nra;
  L.mem = L.val + 4u * (uint32_t)c.nva;
  L.info = L.mem + 4u * (uint32_t)c.nka;
  L.sig = L.info + nset;
  L.total = L.sig + 4u * (uint32_t)c.nsa;
  L.s_info = 0;
  L.s_R = nset;
  L.s_avg = L.s_R + 8u * (uint32_t)c.nsa;
  L.s_total = L.s_avg + 8u * (uint32_t)c.nsa;
  return L;
}

__host__ __device__ inline bool stream_fits(const StreamLayout &L) {
  return L.total <= (uint32_t)kStreamStageBytes && L.s_total <= (uint32_t)kStreamSideBytes;
}

// A chance chunk's stage: the children's values, then its entries of the
// three chance arrays (nothing in the side slot).
struct ChanceLayout {
  uint32_t vb, nch, vs, total;  // offsets of ch_vb, ch_nch, ch_vs entries; bytes
};

__host__ __device__ inline ChanceLayout chance_layout(const StreamChunk &c) {
  ChanceLayout L;
  L.vb = 4u * (uint32_t)c.nva;
  L.nch = L.vb + 4u * (uint32_t)c.nka;
  L.vs = L.nch + 4u * (uint32_t)c.nka;
  L.total = L.vs + 4u * (uint32_t)c.nka;
  return L;
}

__host__ __device__ inline bool chance_fits(const StreamChunk &c) {
  return c.nva > 0 && c.nka > 0 && c.I1 > c.I0 && chance_layout(c).total <= (uint32_t)kStreamStageBytes;
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
    if (clock64() - t0 > 2000000000ll) break;  // about a second at the boost clock
  }
  return false;
}

// Issues the copies of chunk d into a stage and a side slot (one thread):
// the stage's copies counted on its mbarrier bar, the side slot's on sbar (a
// chance chunk puts nothing in the side slot: its phase of sbar completes
// with no bytes). Returns false (and issues nothing) if the chunk does not
// fit. parts: kIssueRest the expected byte counts and every copy but the
// children's values, kIssueValues the children's values (of everything a
// backward launch reads, the one input the backward launch before it
// writes).
constexpr int kIssueRest = 1, kIssueValues = 2, kIssueAll = 3;
__device__ __forceinline__ bool stream_issue(const StreamChunk &d, unsigned char *stage, unsigned char *side,
                                             uint32_t bar, uint32_t sbar, const float2 *reach, const float *v,
                                             const int32_t *mem_vs, const SetInfo *info, const float *sigma,
                                             const double *R, const double *avg, const GameView &g, int parts) {
  if (d.kind == kChunkChance) {
    if (!chance_fits(d)) return false;
    const ChanceLayout C = chance_layout(d);
    const uint32_t s = smem_u32(stage);
    if (parts & kIssueRest) {
      mbar_expect_tx(sbar, 0);  // nothing in the side slot: its phase completes at once
      mbar_expect_tx(bar, C.total);  // the four sizes below add up to this
      bulk_g2s(s + C.vb, g.ch_vb + d.ka, C.nch - C.vb, bar);
      bulk_g2s(s + C.nch, g.ch_nch + d.ka, C.vs - C.nch, bar);
      bulk_g2s(s + C.vs, g.ch_vs + d.ka, C.total - C.vs, bar);
    }
    if (parts & kIssueValues) bulk_g2s(s, v + d.va, C.vb, bar);
    return true;
  }
  if (d.kind != kChunkSets) return false;
  const StreamLayout L = stream_layout(d);
  if (!stream_fits(L) || d.nra <= 0 || d.nva <= 0 || d.nka <= 0 || d.I1 <= d.I0 || d.nsa <= 0) return false;
  const uint32_t s = smem_u32(stage), t = smem_u32(side);
  if (parts & kIssueRest) {
    mbar_expect_tx(sbar, L.s_total);  // the side slot's three copies
    bulk_g2s(t + L.s_info, info + d.I0, L.s_R - L.s_info, sbar);
    bulk_g2s(t + L.s_R, R + d.sa, L.s_avg - L.s_R, sbar);
    bulk_g2s(t + L.s_avg, avg + d.sa, L.s_total - L.s_avg, sbar);
    mbar_expect_tx(bar, L.total);  // the stage's five copies
    bulk_g2s(s + L.reach, reach + d.ra, L.val - L.reach, bar);
    bulk_g2s(s + L.mem, mem_vs + d.ka, L.info - L.mem, bar);
    bulk_g2s(s + L.info, info + d.I0, L.sig - L.info, bar);
    bulk_g2s(s + L.sig, sigma + d.sa, L.total - L.sig, bar);
  }
  if (parts & kIssueValues) bulk_g2s(s + L.val, v + d.va, L.mem - L.val, bar);
  return true;
}

// The member work of one group of sets (G = 1 or 4) of a staged chunk, by
// the kStreamCompute compute threads: thread t serves set j = t % G and
// members t / G, t / G + kStreamCompute / G, ...; writes each member's value and leaves
// the thread's partial regret and average sums, finished by a butterfly over
// the warp's lanes that serve the same set, in racc / macc.
template <int MAXA>
__device__ __forceinline__ void stream_members(const StreamChunk &d, const StreamLayout &L, const unsigned char *stage,
                                               int32_t I, int G, float *v, float (&racc)[MAXA],
                                               float (&macc)[MAXA]) {
  const int tid = threadIdx.x;
  const SetInfo *sinfo = reinterpret_cast<const SetInfo *>(stage + L.info);
  const int gs = G == 4 ? 2 : 0;
  const int j = tid & (G - 1);
  const int LPS = kStreamCompute >> gs;
  const SetInfo si = sinfo[I + j - d.I0];
  const bool p2 = (si.flags >> 8) & 1;
  const float2 *sr = reinterpret_cast<const float2 *>(stage + L.reach);
  const float *sv = reinterpret_cast<const float *>(stage + L.val);
  const int32_t *sm = reinterpret_cast<const int32_t *>(stage + L.mem);
  const float *ss = reinterpret_cast<const float *>(stage + L.sig);
  float sig[MAXA];
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
    const int32_t cb = cbase + q;  // child a at cb + a * nm (action-major block)
    float vc[MAXA];
    float vh = 0.f;
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      if (a < si.na) {
        vc[a] = sv[cb + a * si.nm];
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
#pragma unroll
  for (int a = 0; a < MAXA; ++a) {
    for (int off = G; off < 32; off <<= 1) {
      racc[a] += __shfl_xor_sync(0xffffffffu, racc[a], off);
      macc[a] += __shfl_xor_sync(0xffffffffu, macc[a], off);
    }
  }
}

// The slot update of one group by the update warp: lane = a * G + j
// updates slot a of set j (the warps' partial sums added in warp order),
// then writes sigma^{t+1} of the group's sets.
template <int MAXA>
__device__ __forceinline__ void stream_update(const StreamChunk &d, const StreamLayout &L, const unsigned char *side,
                                              int32_t I, int G, float *sigma, double *Rg, double *avgg, double wt,
                                              int rule, int upd, const float (*red)[4][2 * MAXA]) {
  const int lane = threadIdx.x & 31;
  const SetInfo *sinfo = reinterpret_cast<const SetInfo *>(side + L.s_info);
  const int gs = G == 4 ? 2 : 0;
  const int jj = lane & (G - 1), a = lane >> gs;
  const SetInfo sj = sinfo[I + jj - d.I0];
  const bool q2 = (sj.flags >> 8) & 1;
  const bool live = a < MAXA && a < sj.na && (upd & (q2 ? 2 : 1));
  float pf = 0.f;
  if (live) {
    float r = 0.f, m = 0.f;
    for (int w = 0; w < kStreamWarps; ++w) {  // warps in order
      r += red[w][jj][a];
      m += red[w][jj][MAXA + a];
    }
    const int32_t qs = sj.sb + a;
    const double *sR = reinterpret_cast<const double *>(side + L.s_R);
    const double *sA = reinterpret_cast<const double *>(side + L.s_avg);
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
  if (live) sigma[sj.sb + a] = tot > 0.f ? pf / tot : 1.f / (float)sj.na;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The compute threads' work on a staged chance chunk: thread t sums the
// children of nodes I0 + t, I0 + t + kStreamCompute, ... left to right (as
// bwd_chance does: the same value bit for bit) and writes the node's value.
__device__ __forceinline__ void stream_chance_chunk(const StreamChunk &d, const unsigned char *stage, float *v) {
  const ChanceLayout C = chance_layout(d);
  const float *sv = reinterpret_cast<const float *>(stage);
  const int32_t *svb = reinterpret_cast<const int32_t *>(stage + C.vb);
  const int32_t *snc = reinterpret_cast<const int32_t *>(stage + C.nch);
  const int32_t *svs = reinterpret_cast<const int32_t *>(stage + C.vs);
  for (int32_t i = d.I0 + (int32_t)threadIdx.x; i < d.I1; i += kStreamCompute) {
    const int32_t k = i - d.ka;
    const float *p = sv + (svb[k] - d.va);
    const int32_t n = snc[k];
    float sum = 0.f;
    for (int32_t c = 0; c < n; ++c) sum = sum + p[c];
    v[svs[k]] = sum;
  }
}

// Threads of a streaming CTA: kStreamCompute compute threads, the copy warp
// (its first lane issues every bulk copy) and the update warp (the slot
// updates).
constexpr int kStreamThreads = kStreamCompute + 64;

// Grid: the streaming CTAs over chunks [c0, c1) of this depth (its set
// chunks, then its chance chunks; a depth with wide chance nodes does not
// stream). Chunk i of a CTA uses stage i % kStreamStages (the compute
// threads' data) and side slot i % kStreamSideSlots (set records, R and
// average for the update warp). Barriers of a streaming CTA (every wait
// bounded):
//   full[s]   the copies of the chunk in stage s have landed (bytes counted)
//   empty[s]  the compute threads are done with stage s
//   sfull[k]  the copies of the chunk in side slot k have landed
//   sfree[k]  the update warp is done with side slot k
//   rfull[p]  the compute threads have written the partial sums red[p]
//   rempty[p] the update warp has consumed red[p]
// The copy warp refills stage s with chunk i + kStreamStages as soon as the
// compute threads are done with chunk i and the update warp is done with
// the side slot's previous chunk; the compute warps never wait for a slot
// update, and the update warp, which works through the chunks in order,
// never holds up a refill of a stage. Each barrier's phases are waited for
// in order and a phase cannot complete twice before its waiter sees it: a
// stage is refilled only after its chunk was consumed, a side slot only
// after the update warp released it.
template <int MAXA>
__global__ void __launch_bounds__(kStreamThreads, 2)
    bwd_stream_kernel(GameView g, StateView<float> st, const SetInfo *info, const StreamChunk *chunks, int32_t c0,
                      int32_t c1, int rule, int upd, int *err, int early) {
  static_assert(kStreamSideSlots >= 2 * kStreamStages, "side slots must outlast the stages by a full ring");
  constexpr int S = kStreamStages, K = kStreamSideSlots;
  extern __shared__ __align__(128) unsigned char s_stage[];  // stages, then side slots
  __shared__ __align__(8) uint64_t s_full[S], s_empty[S], s_sfull[K], s_sfree[K], s_rfull[2], s_rempty[2];
  __shared__ StreamChunk s_desc[S], s_sdesc[K];
  __shared__ float s_red[2][kStreamWarps][4][2 * MAXA];
  if (!early) pdl_enter();
  const int32_t b = (int32_t)blockIdx.x;
  const int32_t nb = (int32_t)gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31;
  const int role = tid < kStreamCompute ? 0 : (tid < kStreamCompute + 32 ? 1 : 2);  // compute, copy, update
  const bool producer = tid == kStreamCompute;
  unsigned char *s_side = s_stage + S * kStreamStageBytes;
  if ((smem_u32(s_stage) & 15u) != 0u) {  // bulk copies need 16-byte aligned destinations
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  auto issue = [&](int32_t i, const StreamChunk &dsc, int parts) {
    const int s = i % S, k = i % K;
    if (parts & kIssueRest) {  // before the copies whose barriers publish them
      s_desc[s] = dsc;
      s_sdesc[k] = dsc;
    }
    return stream_issue(dsc, s_stage + s * kStreamStageBytes, s_side + k * kStreamSideBytes, smem_u32(&s_full[s]),
                        smem_u32(&s_sfull[k]), st.reach, st.v, g.mem_vs, info, st.sigma, st.R, st.avg, g, parts);
  };
  int32_t issued = 0;  // chunks issued (copy thread)
  if (producer) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&s_full[s]), 1);
      mbar_init(smem_u32(&s_empty[s]), kStreamCompute);
    }
    for (int k = 0; k < K; ++k) {
      mbar_init(smem_u32(&s_sfull[k]), 1);
      mbar_init(smem_u32(&s_sfree[k]), 32);
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(smem_u32(&s_rfull[p]), kStreamCompute);
      mbar_init(smem_u32(&s_rempty[p]), 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // the first chunks of this CTA. early: the launch before this one is
    // the backward launch of the next depth, which writes only values of
    // this depth's children (and its own slots), so everything else is
    // copied before waiting for that launch to finish (programmatic
    // dependent launch), and the children's values after
    for (int i = 0; i < S; ++i) {
      const int32_t c = c0 + b + i * nb;
      if (c >= c1) break;
      if (!issue(i, chunks[c], early ? kIssueRest : kIssueAll)) {
        atomicExch(err, 1);  // a chunk larger than a stage: never issued, every wait below gives up
        break;
      }
      ++issued;
    }
    if (early) {
      pdl_enter();
      for (int i = 0; i < issued; ++i) issue(i, chunks[c0 + b + i * nb], kIssueValues);
    }
  }
  if (early && !producer) pdl_enter();
  __syncthreads();  // barriers initialised, first copies issued (the only CTA-wide barrier)

  if (role == 1) {
    if (!producer) return;
    // fault-injection hook (err[1], set on the host): issue nothing more, so
    // the other roles' bounded waits for the next chunk run out; the chunks
    // already issued land and are consumed before the CTA leaves
    if (reinterpret_cast<volatile const int *>(err)[1] != 0) return;
    // refill stage i % S with chunk i + S once chunk i is consumed and the
    // side slot's previous chunk released
    int32_t seen = 0;  // chunks known to have landed
    bool ok = issued == S || c0 + b + issued * nb >= c1;
    for (int32_t i = 0; ok; ++i) {
      const int32_t cn = c0 + b + (i + S) * nb;
      if (cn >= c1) break;
      const StreamChunk nd = chunks[cn];  // its latency overlaps the waits
      const int s = i % S;
      if (!mbar_wait(smem_u32(&s_empty[s]), (uint32_t)((i / S) & 1))) { ok = false; break; }
      seen = i + 1;
      const int32_t j = i + S - K;  // the side slot's previous chunk
      if (j >= 0 && !mbar_wait(smem_u32(&s_sfree[(i + S) % K]), (uint32_t)((j / K) & 1))) { ok = false; break; }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (!issue(i + S, nd, kIssueAll)) { ok = false; break; }
      issued = i + S + 1;
    }
    if (!ok) {
      atomicExch(err, 1);
      // let every copy in flight land before the thread leaves (bounded):
      // the last chunks issued into each stage and side slot
      for (int32_t i = max(seen, issued - S); i < issued; ++i)
        mbar_wait(smem_u32(&s_full[i % S]), (uint32_t)((i / S) & 1));
      for (int32_t i = max(0, issued - K); i < issued; ++i)
        mbar_wait(smem_u32(&s_sfull[i % K]), (uint32_t)((i / K) & 1));
    }
    return;
  }

  if (role == 2) {
    const double wt = avg_weight(*st.t + 1, rule);
    int32_t grp = 0;  // groups done by this CTA (selects red[grp & 1] and the barrier phases)
    for (int32_t i = 0;; ++i) {
      const int32_t c = c0 + b + i * nb;
      if (c >= c1) break;
      const int k = i % K;
      if (!mbar_wait(smem_u32(&s_sfull[k]), (uint32_t)((i / K) & 1))) {
        atomicExch(err, 1);
        return;
      }
      const StreamChunk d = s_sdesc[k];  // written before the side slot's copies were issued
      if (d.kind == kChunkSets) {
        const StreamLayout L = stream_layout(d);
        const unsigned char *side = s_side + k * kStreamSideBytes;
        const SetInfo *sinfo = reinterpret_cast<const SetInfo *>(side + L.s_info);
        for (int32_t I = d.I0; I < d.I1; ++grp) {
          const int G = sinfo[I - d.I0].flags & 7;
          const int p = grp & 1;
          if (!mbar_wait(smem_u32(&s_rfull[p]), (uint32_t)((grp >> 1) & 1))) {
            atomicExch(err, 1);
            return;
          }
          stream_update<MAXA>(d, L, side, I, G, st.sigma, st.R, st.avg, wt, rule, upd, s_red[p]);
          mbar_arrive(smem_u32(&s_rempty[p]));
          I += G;
        }
      }
      mbar_arrive(smem_u32(&s_sfree[k]));
    }
    return;
  }

  int32_t grp = 0;
  for (int32_t i = 0;; ++i) {
    const int32_t c = c0 + b + i * nb;
    if (c >= c1) break;
    const int s = i % S;
    if (!mbar_wait(smem_u32(&s_full[s]), (uint32_t)((i / S) & 1))) {
      atomicExch(err, 1);
      return;
    }
    const StreamChunk d = s_desc[s];
    const unsigned char *stage = s_stage + s * kStreamStageBytes;
    if (d.kind == kChunkChance) {
      stream_chance_chunk(d, stage, st.v);
      mbar_arrive(smem_u32(&s_empty[s]));
      continue;
    }
    const StreamLayout L = stream_layout(d);
    const SetInfo *sinfo = reinterpret_cast<const SetInfo *>(stage + L.info);
    for (int32_t I = d.I0; I < d.I1; ++grp) {
      const int G = sinfo[I - d.I0].flags & 7;
      const int p = grp & 1;
      float racc[MAXA], macc[MAXA];
      stream_members<MAXA>(d, L, stage, I, G, st.v, racc, macc);
      // red[p] is free once the update warp consumed it two groups ago
      if (grp >= 2 && !mbar_wait(smem_u32(&s_rempty[p]), (uint32_t)(((grp >> 1) & 1) ^ 1u))) {
        atomicExch(err, 1);
        return;
      }
      if (lane < G) {
#pragma unroll
        for (int a = 0; a < MAXA; ++a) {
          s_red[p][tid >> 5][lane][a] = racc[a];
          s_red[p][tid >> 5][lane][MAXA + a] = macc[a];
        }
      }
      mbar_arrive(smem_u32(&s_rfull[p]));
      if (I + G >= d.I1) mbar_arrive(smem_u32(&s_empty[s]));  // this thread is done with stage s
      I += G;
    }
  }
  // every chunk issued was waited on (full[s]) by the compute threads and
  // (sfull[k]) by the update warp before they left
}

}  // namespace cfr
