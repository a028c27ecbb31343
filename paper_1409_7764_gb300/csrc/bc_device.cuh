// Device helpers shared by the kernel translation units of the GB300
// betweenness-centrality library: L2-coherent loads, a time-bounded grid
// barrier, saturating path-count adds, chunk arrival tickets, warp helpers and
// the optional per-step trace.
#pragma once

#include "bc_internal.cuh"

namespace bcgpu {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ void set_err(Ctl *ctl, int code) { atomicCAS(&ctl->err, 0, code); }

__device__ __forceinline__ int read_err(const Ctl *ctl) {
  return *reinterpret_cast<const volatile int *>(&ctl->err);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// wait is bounded by timeout_ns; on expiry the CTA records KERR_TIMEOUT and
// continues, and every CTA then leaves the kernel at its next error check.
// When snap_dst is given, the last CTA to arrive copies the queue tail there
// before releasing the others: once every CTA has arrived no enqueue of the
// finished level can still be in flight, so the copy is that level's final
// end, and unlike the live tail (which the next level's enqueues advance) it
// reads the same in every CTA.  Returns false when the job is in an error
// state.  `count` CTAs take part (0: the whole grid; a group of CTAs that
// shares a control block otherwise).
__device__ bool grid_sync(Ctl *ctl, long long timeout_ns, int64_t *snap_dst = nullptr,
                          unsigned count = 0) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *genp = &ctl->bar_gen;
    const unsigned gen = *genp;
    __threadfence();
    const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == (count ? count : gridDim.x) - 1) {
      if (snap_dst) *snap_dst = (int64_t)atomicAdd(&ctl->tail, 0ull);
      ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (*genp == gen) {
        if (read_err(ctl)) break;
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
          set_err(ctl, KERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return read_err(ctl) == 0;
}

// ---------------------------------------------------------------------------
// batched kernel: up to 64 sources, bitset frontiers
// ---------------------------------------------------------------------------

template <typename DT> __device__ __forceinline__ DT u64_to(uint64_t x);
template <> __device__ __forceinline__ float u64_to<float>(uint64_t x) {
  // counts below 2^32 (all but pathological graphs) take the 32-bit
  // conversion; both round to nearest, so the value is the same
  return (x >> 32) == 0 ? __uint2float_rn((unsigned)x) : __ull2float_rn(x);
}
template <> __device__ __forceinline__ double u64_to<double>(uint64_t x) { return __ull2double_rn(x); }

// saturating add: on carry the sum pins at 2^64-1 and the flag is raised
__device__ __forceinline__ void sat_add(uint64_t &acc, uint64_t x, bool &ovf) {
  uint64_t s = acc + x;
  if (s < x) {
    s = ~0ull;
    ovf = true;
  }
  acc = s;
}

// Arrival ticket of a heavy-entry chunk: every lane's partial writes are
// fenced, the warp converges, lane 0 takes the ticket, and after the
// broadcast every lane fences again so the last arriver reads all partials.
__device__ __forceinline__ unsigned chunk_ticket(unsigned *arrive, int lane) {
  __threadfence();
  __syncwarp();
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(arrive, 1u);
  t = __shfl_sync(kFull, t, 0);
  __threadfence();
  return t;
}

struct Counters {
  unsigned long long entries = 0, out_e = 0, in_e = 0, dag = 0, reached = 0, heavy = 0;
  unsigned long long busy = 0, idle = 0; // phase clocks (BC_PHASE_CLOCKS builds)
};

#ifndef BC_PHASE_CLOCKS
#define BC_PHASE_CLOCKS 0
#endif
__device__ __forceinline__ long long phase_clock() {
#if BC_PHASE_CLOCKS
  return clock64();
#else
  return 0;
#endif
}



// Optional per-step trace (block 0, thread 0): globaltimer at the start of
// the step, the step's level (negative = backward), items and heavy chunks.
__device__ __forceinline__ void trace_step(const KParams &p, int step, int lvl, int64_t items,
                                           int64_t nhc, int64_t gtid) {
  if (p.trace && gtid == 0 && step < p.trace_cap) {
    unsigned long long *t = p.trace + 4 * (size_t)step;
    t[0] = globaltimer_ns();
    t[1] = (unsigned long long)(long long)lvl;
    t[2] = (unsigned long long)items;
    t[3] = (unsigned long long)nhc;
  }
}

template <typename DT> __device__ __forceinline__ DT warp_sum(DT v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

#ifndef BC_GATHER_UNROLL
#define BC_GATHER_UNROLL 4 // DAG edges gathered per round (lanes-per-source form)
#endif

// ---------------------------------------------------------------------------
// Source masks of W 64-bit words (64*W sources per batch).  Lane j owns the
// sources 32*i + j, i = 0 .. 2W-1 ("slot" i); slot i is bit (i&1)*32 + j of
// word i/2.  Per-vertex masks are stored as W consecutive words.
// ---------------------------------------------------------------------------
template <int W> struct Mask {
  uint64_t w[W];
  __device__ __forceinline__ static Mask zero() {
    Mask m;
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = 0;
    return m;
  }
  __device__ __forceinline__ bool any() const {
    uint64_t a = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) a |= w[i];
    return a != 0;
  }
  __device__ __forceinline__ int popc() const {
    int c = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) c += __popcll(w[i]);
    return c;
  }
  __device__ __forceinline__ bool has(int slot, int lane) const {
    return (w[slot >> 1] >> ((slot & 1) * 32 + lane)) & 1ull;
  }
  __device__ __forceinline__ Mask operator&(const Mask &o) const {
    Mask m;
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = w[i] & o.w[i];
    return m;
  }
  __device__ __forceinline__ Mask operator|(const Mask &o) const {
    Mask m;
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = w[i] | o.w[i];
    return m;
  }
  __device__ __forceinline__ Mask and_not(const Mask &o) const {
    Mask m;
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = w[i] & ~o.w[i];
    return m;
  }
};

// Mask of vertex v from an array of S-word masks (its first W words), through
// L2 (16-byte loads for W >= 2).  S > W: a batch of fewer sources run in a
// workspace laid out for wider ones (the unused words stay zero).
template <int W, int S = W>
__device__ __forceinline__ Mask<W> load_mask(const uint64_t *base, int64_t v) {
  Mask<W> m;
  const uint64_t *q = base + (size_t)v * S;
  if constexpr (W == 1) {
    m.w[0] = ldcg(q);
  } else {
#pragma unroll
    for (int i = 0; i < W; i += 2) {
      const ulonglong2 t = __ldcg(reinterpret_cast<const ulonglong2 *>(q + i));
      m.w[i] = t.x;
      m.w[i + 1] = t.y;
    }
  }
  return m;
}

template <int W, int S = W>
__device__ __forceinline__ void store_mask(uint64_t *base, int64_t v, const Mask<W> &m) {
  uint64_t *q = base + (size_t)v * S;
#pragma unroll
  for (int i = 0; i < W; ++i) q[i] = m.w[i];
}

template <int W, int S = W> __device__ __forceinline__ void zero_mask(uint64_t *base, int64_t v) {
  store_mask<W, S>(base, v, Mask<W>::zero());
}


// Edges whose predecessor rows a warp gathers per round: 8 row loads per
// lane in flight whatever the mask width.
template <int W> struct GatherUnroll {
  static constexpr int value = W == 1 ? BC_GATHER_UNROLL : (W == 2 ? 2 : 1);
};

#ifndef BC_GATHER_FORM
#define BC_GATHER_FORM 1 // 1: carry-counting adds, 32-bit lane tests, 4-byte rows twice as deep
#endif

// Edges per round of the dependency-coefficient gather: as many as keep 8
// 8-byte (16 4-byte) values per lane in flight.
#ifndef BC_NARROW_UNROLL
#define BC_NARROW_UNROLL 2 // edges in flight of 4-byte gathers, relative to 8-byte ones
#endif
#ifndef BC_NARROW_UNROLL_W4
#define BC_NARROW_UNROLL_W4 3 // 4-byte gathers of 256-source batches: edges per round
#endif
template <int W> struct NarrowUnroll {
  static constexpr int value = W == 4 ? BC_NARROW_UNROLL_W4 : BC_NARROW_UNROLL * GatherUnroll<W>::value;
};
template <int W, typename DT> struct CoeffUnroll {
  static constexpr int value = (BC_GATHER_FORM >= 1 && sizeof(DT) == 4)
                                   ? NarrowUnroll<W>::value
                                   : GatherUnroll<W>::value;
};

// Per-warp staging of a gather round's edge masks ([warp][entry][word], see
// RoundList).
__shared__ uint64_t g_mask_stage[kWarpsPerBlock][kWarp][kMaxWords];

// Per-warp list of a gather round's edges that carry sources (non-empty
// mask), packed in lane order: the lane holding such an edge writes its
// vertex and mask at its rank among them, and every lane then reads entry i
// with broadcast shared-memory loads: no search of the ballot for the i-th
// edge's lane and no shuffle of its vertex.  Entries from cnt on read as
// vertex 0 with an empty mask (they gather nothing).
__shared__ int32_t g_vert_stage[kWarpsPerBlock][kWarp];

template <int W> struct RoundList {
  const uint64_t *stg;
  const int32_t *vst;
  int cnt;
  __device__ __forceinline__ RoundList(const Mask<W> &P, int v, unsigned bal, int lane) {
    uint64_t *row = &g_mask_stage[threadIdx.x >> 5][0][0];
    int32_t *vr = g_vert_stage[threadIdx.x >> 5];
    stg = row;
    vst = vr;
    cnt = __popc(bal);
    __syncwarp();
    if ((bal >> lane) & 1u) {
      const int pos = __popc(bal & lanemask_lt());
      vr[pos] = v;
      if constexpr (W == 1) {
        row[pos * kMaxWords] = P.w[0];
      } else {
#pragma unroll
        for (int i = 0; i < W; i += 2)
          *reinterpret_cast<ulonglong2 *>(row + pos * kMaxWords + i) =
              make_ulonglong2(P.w[i], P.w[i + 1]);
      }
    }
    __syncwarp();
  }
  __device__ __forceinline__ int vert(int i) const { return i < cnt ? vst[i] : 0; }
  __device__ __forceinline__ Mask<W> mask(int i) const {
    Mask<W> m;
    if (i >= cnt) return Mask<W>::zero();
    const uint64_t *e = stg + i * kMaxWords;
    if constexpr (W == 1) {
      m.w[0] = e[0];
    } else {
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(e + j);
        m.w[j] = t.x;
        m.w[j + 1] = t.y;
      }
    }
    return m;
  }
};

// s += x, with the carry out of the top bit added to c (c counts carries).
__device__ __forceinline__ void add_count_carry(uint64_t &s, uint64_t x, unsigned &c) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(s), "+r"(c) : "l"(x));
}
__device__ __forceinline__ void add_count_carry(uint32_t &s, uint32_t x, unsigned &c) {
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(s), "+r"(c) : "r"(x));
}

// Edges per round of the path-count gather: 4-byte counts (the 32-bit
// storage form) keep twice as many edges in flight in the same registers.
template <int W, typename CT> struct CountUnroll {
  static constexpr int value = sizeof(CT) == 4 ? NarrowUnroll<W>::value : GatherUnroll<W>::value;
};

// Path counts over the round's shortest-path edges (lanes whose mask P is not
// empty, in lane order): lane j adds row[32*i + j] of each edge's row for
// every slot i whose bit is set, in edge order.  kExact (64-bit counts): the
// carry of slot i is recorded in bit i of cbits (a carry means the true
// count reached 2^64).  Otherwise cbits only counts carries out of the
// count's width: the caller then takes the exact form (64-bit counts, rare:
// counts near 2^64) or promotes the job to 64-bit counts (32-bit storage).
// `unit` (uniform): every predecessor's count is 1 (level 1 of a simple
// graph), so each set bit adds 1 and no row is loaded.
template <int W, bool kExact = true, typename CT = uint64_t, int S = W>
__device__ __forceinline__ void gather_counts_w(const CT *base, int u, const Mask<W> &P,
                                                int lane, CT (&s)[2 * W], unsigned &cbits,
                                                bool unit = false) {
  constexpr int U = CountUnroll<W, CT>::value;
  const unsigned mybit = 1u << lane;
  unsigned bal = __ballot_sync(kFull, P.any());
  if (!bal) return;
  const RoundList<W> rl(P, u, bal, lane);
  for (int i0 = 0; i0 < rl.cnt; i0 += U) {
    CT x[U][2 * W];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const CT *row = base + (size_t)rl.vert(i0 + i) * (kK * S) + lane;
      const Mask<W> PE = rl.mask(i0 + i);
#pragma unroll
      for (int wi = 0; wi < W; ++wi) {
        const uint64_t PP = PE.w[wi];
        const unsigned lo = (unsigned)PP, hi = (unsigned)(PP >> 32);
        x[i][2 * wi] = (lo & mybit) ? (unit ? CT(1) : ldcg(row + 64 * wi)) : CT(0);
        x[i][2 * wi + 1] = (hi & mybit) ? (unit ? CT(1) : ldcg(row + 64 * wi + 32)) : CT(0);
      }
    }
#pragma unroll
    for (int i = 0; i < U; ++i)
#pragma unroll
      for (int t = 0; t < 2 * W; ++t) {
        if ((kExact || BC_GATHER_FORM == 0) && sizeof(CT) == 8) {
          s[t] += x[i][t];
          cbits |= (s[t] < x[i][t] ? 1u : 0u) << t;
        } else {
          add_count_carry(s[t], x[i][t], cbits);
        }
      }
  }
}

// Dependency coefficients over the round's successor edges, added in edge
// order (a missing edge adds +0, which changes no sum of non-negative terms).
template <int W, typename DT, int LS = W>
__device__ __forceinline__ void gather_coeffs_w(const DT *base, int x, const Mask<W> &S,
                                                int lane, DT (&a)[2 * W]) {
  constexpr int U = CoeffUnroll<W, DT>::value;
  const unsigned mybit = 1u << lane;
  unsigned bal = __ballot_sync(kFull, S.any());
  if (!bal) return;
  const RoundList<W> rl(S, x, bal, lane);
  for (int i0 = 0; i0 < rl.cnt; i0 += U) {
    DT y[U][2 * W];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const DT *row = base + (size_t)rl.vert(i0 + i) * (kK * LS) + lane;
      const Mask<W> SE = rl.mask(i0 + i);
#pragma unroll
      for (int wi = 0; wi < W; ++wi) {
        const uint64_t SS = SE.w[wi];
        const unsigned lo = (unsigned)SS, hi = (unsigned)(SS >> 32);
        y[i][2 * wi] = (lo & mybit) ? ldcg(row + 64 * wi) : DT(0);
        y[i][2 * wi + 1] = (hi & mybit) ? ldcg(row + 64 * wi + 32) : DT(0);
      }
    }
#pragma unroll
    for (int i = 0; i < U; ++i)
#pragma unroll
      for (int t = 0; t < 2 * W; ++t) a[t] += y[i][t];
  }
}

// Dependency pull over out-edges [eb, ee) of an entry with mask F from the
// level l+1 masks Dn: lane j sums c[x][32*i + j] over successors x whose
// level-(l+1) mask has source 32*i + j, in edge order.
template <int W, typename DT, int LS = W>
__device__ __forceinline__ void batch_pull_delta_w(const KParams &p, const Mask<W> &F, int eb,
                                                   int ee, const uint64_t *Dn, int lane,
                                                   DT (&a)[2 * W]) {
  const DT *cdep = reinterpret_cast<const DT *>(p.w.cdep);
  for (int base = eb; base < ee; base += kWarp) {
    const int e = base + lane;
    int x = 0;
    Mask<W> S = Mask<W>::zero();
    if (e < ee) {
      x = __ldg(p.g.col_idx + e);
      S = load_mask<W, LS>(Dn, x) & F;
    }
    gather_coeffs_w<W, DT, LS>(cdep, x, S, lane, a);
  }
}

// Writes the path counts of entry w (mask F; counts saturated where the carry
// bit is set) and records the overflowing sources in the control block.
// Counts are stored as CT (32-bit counts are below 2^32 here).
template <int W, typename CT, typename AT, int S = W>
__device__ __forceinline__ void batch_store_sigma_w(const KParams &p, int w, const Mask<W> &F,
                                                    const AT (&s)[2 * W], unsigned cbits,
                                                    int lane) {
  CT *row = reinterpret_cast<CT *>(p.w.sigma) + (size_t)w * (kK * S);
  if constexpr (sizeof(CT) == 4) {
    // 32-bit counts never saturate (a count of 2^32 or more promotes the
    // job to 64-bit counts before it is stored): no carry bits to record
#pragma unroll
    for (int i = 0; i < 2 * W; ++i)
      if (F.has(i, lane)) row[32 * i + lane] = CT(s[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 2 * W; ++i)
      if (F.has(i, lane)) row[32 * i + lane] = ((cbits >> i) & 1u) ? CT(~0ull) : CT(s[i]);
#pragma unroll
    for (int wi = 0; wi < W; ++wi) {
      const uint64_t ob = ((uint64_t)__ballot_sync(kFull, (cbits >> (2 * wi)) & 1u) |
                           ((uint64_t)__ballot_sync(kFull, (cbits >> (2 * wi + 1)) & 1u) << 32)) &
                          F.w[wi];
      if (ob && lane == 0) atomicOr(&p.w.ctl->ovf[wi], (unsigned long long)ob);
    }
  }
}

// Last heavy entry h in [base, base+cnt) whose first chunk hq_c[h] <= item:
// a 32-ary search (each round the lanes probe 32 evenly spaced entries), so
// a level with up to 32^3 heavy entries needs at most three L2 round trips.
// hq_c strictly increases with h and hq_c[base] == 0.
__device__ int64_t warp_find_heavy(const int64_t *hq_c, int64_t base, int64_t cnt, int64_t item,
                                   int lane) {
  int64_t lo = 0, hi = cnt;
  while (hi - lo > 1) {
    const int64_t span = hi - lo;
    if (span <= kWarp) {
      bool ok = false;
      if (lane < span) ok = ldcg(hq_c + base + lo + lane) <= item;
      const unsigned b = __ballot_sync(kFull, ok);
      return base + lo + (31 - __clz(b));
    }
    const int64_t idx = lo + span * lane / kWarp;
    const bool ok = ldcg(hq_c + base + idx) <= item;
    const unsigned b = __ballot_sync(kFull, ok);
    const int t = 31 - __clz(b);
    const int64_t nlo = lo + span * t / kWarp;
    const int64_t nhi = (t == kWarp - 1) ? hi : lo + span * (t + 1) / kWarp;
    lo = nlo;
    hi = nhi;
  }
  return base + lo;
}

} // namespace
} // namespace bcgpu
