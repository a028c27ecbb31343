// Batched sweeps of the GB300 exact betweenness-centrality library, shared by
// the kernel translation units.
//
// Both kernels run Brandes' two sweeps (paper, Section I; the GPU designs it
// studies are in Section II.A) as ONE persistent cooperative launch per
// batch of sources, with levels separated by a software grid barrier whose
// waits are bounded in time:
//
//   forward step l  (one barrier per level)
//     - every frontier entry w of level l pulls its path counts from its
//       in-neighbours at level l-1:  sigma[w] = sum sigma[u]   (no atomics);
//     - and pushes discovery to its out-neighbours: bits new to a vertex x
//       are OR-ed into visited[x] and into the dense next-level mask, and x
//       is appended to the level-(l+1) queue on its first touch;
//   backward step l (one barrier per level, l = L-1 .. 0)
//     - every entry v of level l pulls from its successors x (edge v->x with
//       x one level deeper for that source):
//           delta[v] = sigma[v] * sum c[x],   c[x] = (1 + delta[x]) / sigma[x]
//       which is Brandes' dependency sum with sigma[v] factored out; no
//       atomics on delta, fixed reduction order, so results are
//       deterministic;
//     - BC[v] += sum over sources j with s_j != v of delta_j[v].
//
// The batched kernel advances up to 64 sources together: frontiers and
// visited sets are u64 bitsets (bit j = source j), per-vertex state is laid
// out source-innermost ([n][64]) so a warp touches one contiguous row, lane
// j owning sources j and j+32.  The plain kernel is the one-source baseline
// (the paper's multi-block-per-source design, Section II.A, with the level
// loop moved on-device), lanes spread over edges.
//
// Work inside a level is balanced dynamically: warps fetch small groups of
// items from a per-step counter.  High-degree vertices (in+out degree >
// kChunk) are split into chunks that different warps process; partial sums
// meet in scratch and the last arriving warp (ticket counter) reduces them in
// chunk order, which keeps the result deterministic.  Memory written during a launch by another SM is
// always read through L2 (ld.global.cg), never a possibly stale L1 line.
#pragma once

#include "bc_device.cuh"

namespace bcgpu {
namespace {


struct LevelView {
  int lvl;
  int64_t lo, hi;        // queue range of this level
  int64_t hoff;          // first heavy entry of this level
  int64_t nheavy;        // heavy entries of this level
  int64_t nhc;           // heavy chunks of this level
  int64_t hoff_next;     // first heavy entry of the next level (forward)
};

// Warp-aggregated append of newly discovered vertices to the next level.
__device__ __forceinline__ void enqueue_new(const KParams &p, const LevelView &lv, bool isnew,
                                            int x, int lane) {
  const unsigned bal = __ballot_sync(kFull, isnew);
  if (!bal) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&p.w.ctl->tail, (unsigned long long)__popc(bal));
  base = __shfl_sync(kFull, base, 0);
  if (!isnew) return;
  const long long pos = (long long)base + __popc(bal & lanemask_lt());
  if (pos >= p.w.cap) {
    set_err(p.w.ctl, KERR_QUEUE);
    return;
  }
  p.w.qv[pos] = x;
  const int nch = __ldg(p.g.nchunks + x);
  if (nch > 0) {
    const unsigned long long h =
        atomicAdd(&p.w.hpack[lv.lvl + 1], (1ull << 32) | (unsigned long long)nch);
    const int64_t hidx = lv.hoff_next + (int64_t)(h >> 32);
    const int64_t cpre = (int64_t)(h & 0xffffffffull);
    if (hidx >= p.w.hcap) {
      set_err(p.w.ctl, KERR_HEAVY);
      return;
    }
    if (cpre + nch > p.w.chunk_cap) {
      set_err(p.w.ctl, KERR_CHUNKS);
      return;
    }
    p.w.hq_e[hidx] = pos;
    p.w.hq_c[hidx] = cpre;
  }
}

// ---- step work distribution ------------------------------------------------
//
// The work of one step is a list of items: the chunks of the level's heavy
// entries first (largest units first), then its light entries.  Warps take
// `grab` consecutive items (KParams::grab) per fetch from the step's counter and fetch the
// next group before processing the current one, so the counter round trip
// overlaps useful work.

// The first group of every warp is static (items gwarp*grab ..), so a step
// whose items all fit in one group per warp touches no counter; later groups
// come from the step's counter.
__device__ __forceinline__ int64_t next_items(unsigned long long *ctr, int64_t total,
                                              int64_t stat, int grab, int lane) {
  if (total <= stat) return total;
  unsigned long long v = 0;
  if (lane == 0) v = atomicAdd(ctr, (unsigned long long)grab);
  return stat + (int64_t)__shfl_sync(kFull, v, 0);
}

// Tracks the heavy entry of consecutive chunk items within one warp.
struct HeavyCursor {
  int64_t h = -1;
  int first = 0, end = 0;
  __device__ __forceinline__ void seek(const KParams &p, const LevelView &lv, int64_t item,
                                       int lane) {
    if (h >= 0 && item >= first && item < end) return;
    if (h >= 0 && item == end && h + 1 < lv.hoff + lv.nheavy) {
      ++h;
    } else {
      h = warp_find_heavy(p.w.hq_c, lv.hoff, lv.nheavy, item, lane);
    }
    first = (int)ldcg(p.w.hq_c + h);
    end = (int)((h + 1 < lv.hoff + lv.nheavy) ? ldcg(p.w.hq_c + h + 1) : lv.nhc);
  }
};

__device__ __forceinline__ void zero_ring_ahead(Ctl *ctl, int step, int64_t gtid) {
  if (gtid == 0) ctl->work[(step + 2) & 3] = 0;
}

constexpr int kStage = 64; // per-warp staging of newly discovered vertices

// Adds the in- and out-degrees of a level's new vertices (summed over the
// warp) to that level's totals, which choose the direction of the level's
// path-count step.
__device__ __forceinline__ void add_level_degrees(const KParams &p, int lvl,
                                                  unsigned long long din,
                                                  unsigned long long dout, int lane) {
  din = warp_sum_u64(din);
  dout = warp_sum_u64(dout);
  if (lane == 0 && (din | dout)) {
    atomicAdd(p.w.lsum + 2 * lvl, din);
    atomicAdd(p.w.lsum + 2 * lvl + 1, dout);
  }
}

// Appends a warp's staged vertices to the next level's queue with one tail
// atomic; high-degree ones also get their chunk range in the level's list.
__device__ __forceinline__ void stage_flush(const KParams &p, const LevelView &lv, const int *buf,
                                            int nst, int lane) {
  if (nst == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&p.w.ctl->tail, (unsigned long long)nst);
  base = __shfl_sync(kFull, base, 0);
  unsigned long long din = 0, dout = 0;
  const bool sums = p.push_ratio != 0;
  for (int i = lane; i < nst; i += kWarp) {
    const long long pos = (long long)base + i;
    if (pos >= p.w.cap) {
      set_err(p.w.ctl, KERR_QUEUE);
      continue;
    }
    const int x = buf[i];
    p.w.qv[pos] = x;
    if (sums) {
      din += (unsigned long long)(__ldg(p.g.in_ptr + x + 1) - __ldg(p.g.in_ptr + x));
      dout += (unsigned long long)(__ldg(p.g.row_ptr + x + 1) - __ldg(p.g.row_ptr + x));
    }
    const int nch = __ldg(p.g.nchunks + x);
    if (nch > 0) {
      const unsigned long long h =
          atomicAdd(&p.w.hpack[lv.lvl + 1], (1ull << 32) | (unsigned long long)nch);
      const int64_t hidx = lv.hoff_next + (int64_t)(h >> 32);
      const int64_t cpre = (int64_t)(h & 0xffffffffull);
      if (hidx >= p.w.hcap) {
        set_err(p.w.ctl, KERR_HEAVY);
        continue;
      }
      if (cpre + nch > p.w.chunk_cap) {
        set_err(p.w.ctl, KERR_CHUNKS);
        continue;
      }
      p.w.hq_e[hidx] = pos;
      p.w.hq_c[hidx] = cpre;
    }
  }
  if (sums) add_level_degrees(p, lv.lvl + 1, din, dout, lane);
}

// Stages the vertices this round discovered first (isnew lanes) in the
// warp's shared buffer; the buffer is flushed to the queue when full and at
// the end of the step.
__device__ __forceinline__ void stage_new(const KParams &p, const LevelView &lv, bool isnew, int x,
                                          int *buf, int &nst, int lane) {
  const unsigned bal = __ballot_sync(kFull, isnew);
  if (!bal) return;
  const int c = __popc(bal);
  if (nst + c > kStage) {
    __syncwarp();
    stage_flush(p, lv, buf, nst, lane);
    __syncwarp();
    nst = 0;
  }
  if (isnew) buf[nst + __popc(bal & lanemask_lt())] = x;
  nst += c;
}

// Path-count pull of an entry (mask F) over its in-edges [ib, ib + din)
// from the level l-1 masks Pm, in edge order (`unit`: level l-1's counts
// are all 1, see gather_counts_w).
template <int W, bool kExact, typename CT, int S = W>
__device__ __forceinline__ void pull_counts(const KParams &p, const Mask<W> &F, int ib, int din,
                                            const uint64_t *Pm, int lane, CT (&s)[2 * W],
                                            unsigned &cbits, unsigned long long &dag,
                                            bool unit) {
  for (int r = 0; r < din; r += kWarp) {
    const int t = r + lane;
    int u = 0;
    Mask<W> P = Mask<W>::zero();
    if (t < din) {
      u = __ldg(p.g.in_idx + ib + t);
      P = load_mask<W, S>(Pm, u) & F;
    }
    dag += P.popc(); // per lane; the warp's counters are summed at the flush
    gather_counts_w<W, kExact, CT, S>(reinterpret_cast<const CT *>(p.w.sigma), u, P, lane, s,
                                      cbits, unit);
  }
}

// The same pull again with every slot's carry recorded, for an entry whose
// fast pull saw a carry (some count reached 2^64): same sums, flags per slot.
template <int W, int S = W>
__device__ __forceinline__ void exact_counts(const KParams &p, const Mask<W> &F, int ib, int din,
                                          const uint64_t *Pm, int lane, uint64_t (&s)[2 * W],
                                          unsigned &cbits, bool unit) {
#pragma unroll
  for (int i = 0; i < 2 * W; ++i) s[i] = 0;
  cbits = 0;
  unsigned long long dag = 0; // counted by the fast pull already
  pull_counts<W, true, uint64_t, S>(p, F, ib, din, Pm, lane, s, cbits, dag, unit);
}

// Pushed path counts (the other direction of the forward step at level l):
// entry u of level l-1 (mask F, its sources at level l-1) adds its counts
// along its out-edges [ob, oe) to every vertex x whose level-l mask A[x]
// shares a source: sigma[x][j] += sigma[u][j] for j in F & A[x].  The masks
// of level l are complete when the step starts, so exactly the
// shortest-path DAG edges into level l receive counts; the adds are 64-bit
// integer atomics, whose order does not change the sums.  The target counts
// start at zero (every batch resets the counts it wrote).  64-bit counts:
// overflow is ruled out before adding: the step refuses (KERR_PUSH, and the
// job reruns pulling counts) as soon as a pushed count is 2^32 or more, so
// every sum of fewer than 2^31 pushed terms stays below 2^63, and the adds
// need no reply.  32-bit counts: each add returns the old value, and a sum
// that wraps promotes the job to 64-bit counts (KERR_WIDE).
__device__ __forceinline__ void push_add(uint64_t *a, uint64_t v, unsigned &) {
  atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)v);
}
__device__ __forceinline__ void push_add(uint32_t *a, uint32_t v, unsigned &wrap) {
  const unsigned old = atomicAdd(reinterpret_cast<unsigned *>(a), v);
  wrap |= (old + v < old) ? 1u : 0u;
}
template <int W, typename CT, int S = W>
__device__ __forceinline__ void push_counts(const KParams &p, int u, const Mask<W> &F, int ob,
                                            int oe, const uint64_t *A, int lane,
                                            unsigned long long &dag) {
  CT own[2 * W];
  const CT *srow = reinterpret_cast<const CT *>(p.w.sigma) + (size_t)u * (kK * S) + lane;
  unsigned big = 0, wrap = 0;
#pragma unroll
  for (int i = 0; i < 2 * W; ++i) {
    own[i] = F.has(i, lane) ? ldcg(srow + 32 * i) : CT(0);
    if constexpr (sizeof(CT) == 8) big |= (unsigned)(own[i] >> 32);
  }
  if (sizeof(CT) == 8 && __any_sync(kFull, big != 0)) {
    set_err(p.w.ctl, KERR_PUSH);
    return;
  }
  const unsigned mybit = 1u << lane;
  for (int r = ob; r < oe; r += kWarp) {
    const int t = r + lane;
    int x = 0;
    Mask<W> P = Mask<W>::zero();
    if (t < oe) {
      x = __ldg(p.g.col_idx + t);
      P = load_mask<W, S>(A, x) & F;
    }
    dag += P.popc(); // per lane; the warp's counters are summed at the flush
    unsigned bal = __ballot_sync(kFull, P.any());
    if (!bal) continue;
    const RoundList<W> rl(P, x, bal, lane);
    for (int i = 0; i < rl.cnt; ++i) {
      CT *row = reinterpret_cast<CT *>(p.w.sigma) + (size_t)rl.vert(i) * (kK * S) + lane;
      const Mask<W> PE = rl.mask(i);
#pragma unroll
      for (int wi = 0; wi < W; ++wi) {
        const uint64_t PP = PE.w[wi];
        if ((unsigned)PP & mybit) push_add(row + 64 * wi, own[2 * wi], wrap);
        if ((unsigned)(PP >> 32) & mybit) push_add(row + 64 * wi + 32, own[2 * wi + 1], wrap);
      }
    }
  }
  if (sizeof(CT) == 4 && __any_sync(kFull, wrap != 0)) set_err(p.w.ctl, KERR_WIDE);
}

// Forward work of one frontier entry (mask F) at level l: the path-count
// pull over in-edges [ib, ie) and the discovery push over out-edges
// [ob, oe).  A vertex x gets the bits F & ~visited[x], OR-ed into its
// level-(l+1) mask and into visited[x] (so visited holds every source that
// reached x at levels up to l+1, and one load tests it), and the first
// toucher of x at level l+1 queues it.  With one mask word the two
// scans advance together, 32 edges of each per round so that their loads
// overlap, and the OR's returned old value (all zero before) tells the first
// toucher; it is read only after the round's path-count gathers.  With
// several words no single atomic covers the mask: a claim on x decides
// (claim[x] < l+2 before, raised to l+2).
// After a fast pull saw a carry: 64-bit counts pull again recording each
// slot's carry (the counts saturate); 32-bit counts stop the batch, and the
// job reruns with 64-bit counts.
template <int W, typename CT, int S = W>
__device__ __forceinline__ void settle_carries(const KParams &p, const Mask<W> &F, int ib,
                                               int din, const uint64_t *Pm, int lane,
                                               CT (&s)[2 * W], unsigned &cbits,
                                               unsigned carries, bool unit) {
  if (!__any_sync(kFull, carries != 0)) return;
  if constexpr (sizeof(CT) == 4) set_err(p.w.ctl, KERR_WIDE);
  else exact_counts<W, S>(p, F, ib, din, Pm, lane, s, cbits, unit);
}

template <int W, typename CT, int S = W>
__device__ __forceinline__ void fwd_scan(const KParams &p, const LevelView &lv, const Mask<W> &F,
                                         int ib, int ie, int ob, int oe,
                                         const uint64_t *A, const uint64_t *Pm, uint64_t *Bn,
                                         int *stage, int &nst, int lane, CT (&s)[2 * W],
                                         unsigned &cbits, unsigned long long &dag,
                                         bool unit = false) {
  const int din = ie > ib ? ie - ib : 0, dout = oe > ob ? oe - ob : 0;
  const int claim_to = lv.lvl + 2;
  constexpr bool kFast = BC_GATHER_FORM >= 1 || sizeof(CT) == 4;
  unsigned carries = 0; // fast form: carries out of the count's width
  if constexpr (W >= 2) {
    // wide masks: the pull and the push run as two loops, so the registers
    // of the path-count gathers and of the discovery masks are not live
    // together
    pull_counts<W, !kFast, CT, S>(p, F, ib, din, Pm, lane, s, kFast ? carries : cbits, dag,
                                  unit);
    if (kFast) settle_carries<W, CT, S>(p, F, ib, din, Pm, lane, s, cbits, carries, unit);
    for (int r = 0; r < dout; r += kWarp) {
      const int t = r + lane;
      int x = 0;
      bool first = false;
      if (t < dout) {
        x = __ldg(p.g.col_idx + ob + t);
        const Mask<W> nb = F.and_not(load_mask<W, S>(p.w.vis, x));
        if (nb.any()) {
          unsigned long long *bx = reinterpret_cast<unsigned long long *>(Bn + (size_t)x * S);
          unsigned long long *vx = reinterpret_cast<unsigned long long *>(p.w.vis + (size_t)x * S);
#pragma unroll
          for (int wi = 0; wi < W; ++wi)
            if (nb.w[wi]) {
              atomicOr(bx + wi, nb.w[wi]);
              atomicOr(vx + wi, nb.w[wi]);
            }
          first = atomicMax(p.w.claim + x, claim_to) < claim_to;
        }
      }
      stage_new(p, lv, first, x, stage, nst, lane);
    }
  } else {
    const int span = din > dout ? din : dout;
    for (int r = 0; r < span; r += kWarp) {
      const int t = r + lane;
      const bool vi = t < din, vo = t < dout;
      int u = 0, x = 0;
      if (vi) u = __ldg(p.g.in_idx + ib + t);
      if (vo) x = __ldg(p.g.col_idx + ob + t);
      uint64_t P = 0, nb = 0;
      if (vi) P = ldcg(Pm + (size_t)u * S) & F.w[0];
      if (vo) nb = F.w[0] & ~ldcg(p.w.vis + (size_t)x * S);
      unsigned long long old = 1;
      if (nb) {
        old = atomicOr(reinterpret_cast<unsigned long long *>(Bn + (size_t)x * S), nb);
        atomicOr(reinterpret_cast<unsigned long long *>(p.w.vis + (size_t)x * S), nb);
      }
      dag += __popcll(P); // per lane; the warp's counters are summed at the flush
      Mask<1> PM;
      PM.w[0] = P;
      gather_counts_w<1, !kFast, CT, S>(reinterpret_cast<const CT *>(p.w.sigma), u, PM, lane, s,
                                        kFast ? carries : cbits, unit);
      stage_new(p, lv, nb != 0 && old == 0, x, stage, nst, lane);
    }
    if (kFast) settle_carries<1, CT, S>(p, F, ib, din, Pm, lane, s, cbits, carries, unit);
  }
}

#ifndef BC_CONTRIB_FORM
#define BC_CONTRIB_FORM 1 // FP32 dependencies: 1 = compensated FP32 pair per entry, 0 = FP64
#endif

// Knuth's error-free sum of two floats: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Sum of the lane's per-source dependencies of one entry over the warp,
// returned to lane 0 as a double.  FP64 dependencies add in FP64.  FP32
// dependencies add as a compensated pair of floats (a two-sum running value
// and its accumulated error, about 46 significant bits for these sums of
// positive terms) and widen once at the end: GB300's FP64 pipe is a small
// fraction of its FP32 one, and an FP64 add per source and entry measured a
// visible share of the kernel.
template <typename DT, int W> struct EntrySum {
  double d = 0.0;
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(DT x) {
    if constexpr (sizeof(DT) == 8 || BC_CONTRIB_FORM == 0) {
      d += (double)x;
    } else {
      float e;
      two_sum(hi, (float)x, hi, e);
      lo += e;
    }
  }
  __device__ __forceinline__ double warp_total() {
    if constexpr (sizeof(DT) == 8 || BC_CONTRIB_FORM == 0) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(kFull, d, off);
      return d;
    } else {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float ohi = __shfl_down_sync(kFull, hi, off);
        const float olo = __shfl_down_sync(kFull, lo, off);
        float e;
        two_sum(hi, ohi, hi, e);
        lo += olo + e;
      }
      return (double)hi + (double)lo;
    }
  }
};

#ifndef BC_FAST_FP32_DIV
#define BC_FAST_FP32_DIV 1
#endif
// The dependency coefficient's division.  FP64: IEEE division.  FP32: the
// fast reciprocal-based division (__fdividef, within 2 ulp for these
// operands: path counts below 2^64 are far from the range where it returns
// 0), about a fifth of the IEEE sequence's instructions; well inside the FP32
// path's error bound (1e-4 relative to exact FP64 dependencies).
__device__ __forceinline__ double coeff_div(double a, double b) { return a / b; }
__device__ __forceinline__ float coeff_div(float a, float b) {
  return BC_FAST_FP32_DIV ? __fdividef(a, b) : a / b;
}

// Batch: closes entry v (mask F) at level l of the backward sweep given the
// lane's successor sums a, its path counts sg and (lane 0) the current BC
// value bcv, all loaded by the caller ahead of the successor scan:
// dependencies, coefficients, BC, resets.  The entry's path counts are
// reset to zero here, so every batch starts on zeroed counts (the pushed
// form of the forward step adds into them).  At level 0 every source bit of
// the entry is the vertex itself, whose own dependency is never added to its
// BC; at deeper levels no source of the entry is the vertex.
template <typename DT, int W, bool SQ, typename CT, int S = W>
__device__ __forceinline__ void batch_finish(const KParams &p, int lvl, int v, const Mask<W> &F,
                                             const DT (&a)[2 * W], const CT (&sg)[2 * W],
                                             double bcv, uint64_t *Wn, int lane) {
  DT *crow = reinterpret_cast<DT *>(p.w.cdep) + (size_t)v * (kK * S);
  CT *srow = reinterpret_cast<CT *>(p.w.sigma) + (size_t)v * (kK * S);
  EntrySum<DT, W> sum;
  double contrib2 = 0.0;
  const int n = p.g.n;
#pragma unroll
  for (int i = 0; i < 2 * W; ++i)
    if (F.has(i, lane)) {
      const int j = 32 * i + lane; // source index within the batch (j < k)
      const DT sf = u64_to<DT>((uint64_t)sg[i]);
      const DT dl = sf * a[i];
      crow[j] = coeff_div(DT(1) + dl, sf);
      srow[j] = 0;
      if (lvl > 0) {
        sum.add(dl);
        if (SQ) contrib2 += (double)dl * (double)dl;
      }
      if (p.dbg_d) {
        const size_t o = (size_t)j * n + v;
        p.dbg_d[o] = lvl;
        p.dbg_sigma[o] = sg[i];
        p.dbg_delta[o] = (double)dl;
      }
    }
  const double contrib = sum.warp_total();
  if (SQ) {
    // squared per-source terms for the sampled-source estimator's variance
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) contrib2 += __shfl_down_sync(kFull, contrib2, off);
    if (lane == 0 && contrib2 != 0.0) p.bc2[v] = ldcg(p.bc2 + v) + contrib2;
  }
  if (lane == 0) {
    if (contrib != 0.0) p.bc[v] = bcv + contrib;
    zero_mask<W, S>(p.w.vis, v);
    if (Wn) store_mask<W, S>(Wn, v, F);
    if (W > 1) p.w.claim[v] = 0;
  }
}

// Loads of an entry's own path counts and BC value, issued before its
// successor scan so they overlap it.
template <int W, typename CT, int S = W> struct EntryOwn {
  CT sg[2 * W];
  double bcv;
  __device__ __forceinline__ EntryOwn(const KParams &p, int v, const Mask<W> &F, int lane) {
    const CT *srow = reinterpret_cast<const CT *>(p.w.sigma) + (size_t)v * (kK * S);
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) sg[i] = F.has(i, lane) ? ldcg(srow + 32 * i + lane) : CT(0);
    bcv = lane == 0 ? ldcg(p.bc + v) : 0.0;
  }
};

// Headers of up to kEntries consecutive queue entries, loaded with one round
// of lane-parallel loads: lane kEntries*f + i holds field f of entry i.
template <int W, int kFields> struct EntryHeaders {
  static constexpr int kEntries = kFields * 4 <= kWarp ? 4 : 2;
  uint64_t hv;
  int cnt;
  __device__ __forceinline__ uint64_t field(int f, int i) const {
    return __shfl_sync(kFull, hv, kEntries * f + i);
  }
  __device__ __forceinline__ Mask<W> mask(int i) const {
    Mask<W> m;
#pragma unroll
    for (int wi = 0; wi < W; ++wi) m.w[wi] = field(wi, i);
    return m;
  }
};

// Forward headers: fields 0..W-1 = mask words (from the dense level mask),
// then in-CSR range, out-CSR range, chunk count, vertex id.
template <int W> struct FwdField {
  static constexpr int kIn0 = W, kIn1 = W + 1, kOut0 = W + 2, kOut1 = W + 3, kNch = W + 4,
                       kId = W + 5, kCount = W + 6;
};
template <int W, int S = W>
__device__ __forceinline__ EntryHeaders<W, FwdField<W>::kCount>
fwd_headers(const KParams &p, const uint64_t *A, int64_t e0, int cnt, int lane) {
  using F = FwdField<W>;
  using H = EntryHeaders<W, F::kCount>;
  if (cnt > H::kEntries) { // more items per fetch than one header round holds
    set_err(p.w.ctl, KERR_GRAB);
    cnt = H::kEntries;
  }
  int wv = 0;
  if (lane < cnt) wv = ldcg(p.w.qv + e0 + lane);
  const int i = lane % H::kEntries, f = lane / H::kEntries;
  const int w = __shfl_sync(kFull, wv, i);
  uint64_t hv = 0;
  if (i < cnt && f < F::kCount) {
    if (f < W) hv = ldcg(A + (size_t)w * S + f);
    else if (f == F::kIn0) hv = (uint64_t)(uint32_t)__ldg(p.g.in_ptr + w);
    else if (f == F::kIn1) hv = (uint64_t)(uint32_t)__ldg(p.g.in_ptr + w + 1);
    else if (f == F::kOut0) hv = (uint64_t)(uint32_t)__ldg(p.g.row_ptr + w);
    else if (f == F::kOut1) hv = (uint64_t)(uint32_t)__ldg(p.g.row_ptr + w + 1);
    else if (f == F::kNch) hv = (uint64_t)(uint32_t)__ldg(p.g.nchunks + w);
    else hv = (uint64_t)(uint32_t)w;
  }
  H h;
  h.hv = hv;
  h.cnt = cnt;
  return h;
}

// Backward headers: fields 0..W-1 = mask words (queue), then out-CSR range,
// chunk count, vertex id.
template <int W> struct BwdField {
  static constexpr int kOut0 = W, kOut1 = W + 1, kNch = W + 2, kId = W + 3, kCount = W + 4;
};
template <int W, int S = W>
__device__ __forceinline__ EntryHeaders<W, BwdField<W>::kCount>
bwd_headers(const KParams &p, int64_t e0, int cnt, int lane) {
  using F = BwdField<W>;
  using H = EntryHeaders<W, F::kCount>;
  if (cnt > H::kEntries) {
    set_err(p.w.ctl, KERR_GRAB);
    cnt = H::kEntries;
  }
  int wv = 0;
  if (lane < cnt) wv = ldcg(p.w.qv + e0 + lane);
  const int i = lane % H::kEntries, f = lane / H::kEntries;
  const int v = __shfl_sync(kFull, wv, i);
  uint64_t hv = 0;
  if (i < cnt && f < F::kCount) {
    if (f < W) hv = ldcg(p.w.qm + (size_t)(e0 + i) * S + f);
    else if (f == F::kOut0) hv = (uint64_t)(uint32_t)__ldg(p.g.row_ptr + v);
    else if (f == F::kOut1) hv = (uint64_t)(uint32_t)__ldg(p.g.row_ptr + v + 1);
    else if (f == F::kNch) hv = (uint64_t)(uint32_t)__ldg(p.g.nchunks + v);
    else hv = (uint64_t)(uint32_t)v;
  }
  H h;
  h.hv = hv;
  h.cnt = cnt;
  return h;
}

// Synchronisation scope of one batch: the whole grid of a cooperative launch
// (levels separated by the time-bounded grid barrier) ...
struct GridScope {
  static constexpr bool kGrid = true;
  __device__ __forceinline__ int rank() const { return (int)blockIdx.x; }
  __device__ __forceinline__ int size() const { return (int)gridDim.x; }
  __device__ __forceinline__ bool sync(Ctl *ctl, long long timeout_ns,
                                       int64_t *snap = nullptr) const {
    return grid_sync(ctl, timeout_ns, snap);
  }
};

// ... or a group of the grid's thread blocks that runs its own batches
// (several batches at once on disjoint sets of SMs; the group's barrier
// counts its blocks on its own workspace's control block) ...
struct GroupScope {
  static constexpr bool kGrid = true;
  int g, gsize;
  __device__ __forceinline__ int rank() const { return (int)blockIdx.x - g * gsize; }
  __device__ __forceinline__ int size() const { return gsize; }
  __device__ __forceinline__ bool sync(Ctl *ctl, long long timeout_ns,
                                       int64_t *snap = nullptr) const {
    return grid_sync(ctl, timeout_ns, snap, (unsigned)gsize);
  }
};

// ... or one thread block that owns the whole batch (CTA barriers; used for
// many small graphs in one launch).  The snapshot of the queue tail is taken
// by thread 0 between two barriers, as the grid barrier's last arriver does.
struct CtaScope {
  static constexpr bool kGrid = false;
  __device__ __forceinline__ int rank() const { return 0; }
  __device__ __forceinline__ int size() const { return 1; }
  __device__ __forceinline__ bool sync(Ctl *ctl, long long, int64_t *snap = nullptr) const {
    __syncthreads();
    if (snap && threadIdx.x == 0)
      *snap = (int64_t)*reinterpret_cast<volatile unsigned long long *>(&ctl->tail);
    __syncthreads();
    return read_err(ctl) == 0;
  }
};

// Sums a warp's per-lane counters and adds them to the job counters.
__device__ __forceinline__ void flush_counters(unsigned long long *job_cnt, Counters cnt,
                                               int lane) {
  cnt.entries = warp_sum_u64(cnt.entries);
  cnt.out_e = warp_sum_u64(cnt.out_e);
  cnt.in_e = warp_sum_u64(cnt.in_e);
  cnt.dag = warp_sum_u64(cnt.dag);
  cnt.reached = warp_sum_u64(cnt.reached);
  cnt.heavy = warp_sum_u64(cnt.heavy);
  if (lane == 0) {
    atomicAdd(job_cnt + CNT_ENTRIES, cnt.entries);
    atomicAdd(job_cnt + CNT_OUT_EDGES, cnt.out_e);
    atomicAdd(job_cnt + CNT_IN_EDGES, cnt.in_e);
    atomicAdd(job_cnt + CNT_DAG, cnt.dag);
    atomicAdd(job_cnt + CNT_REACHED, cnt.reached);
    atomicAdd(job_cnt + CNT_HEAVY, cnt.heavy);
    if (BC_PHASE_CLOCKS) {
      atomicAdd(job_cnt + CNT_BUSY, cnt.busy);
      atomicAdd(job_cnt + CNT_IDLE, cnt.idle);
    }
  }
}

#ifndef BC_OWN_EARLY_MAX_W
#define BC_OWN_EARLY_MAX_W 2 // widest mask whose entries preload their own counts
#endif

// Work counters of one warp of the batch kernels, kept in shared memory
// (lane 0 updates them) so that they hold no registers; the per-lane DAG pair
// count stays in a register.
struct WarpCounters {
  unsigned long long entries, out_e, in_e, reached, heavy, busy, idle;
};

__device__ __forceinline__ void zero_counters(WarpCounters &w, int lane) {
  if (lane == 0) w = WarpCounters{0, 0, 0, 0, 0, 0, 0};
  __syncwarp();
}

__device__ __forceinline__ Counters to_counters(const WarpCounters &w, unsigned long long dag,
                                                int lane) {
  Counters c;
  c.dag = dag;
  if (lane == 0) {
    c.entries = w.entries;
    c.out_e = w.out_e;
    c.in_e = w.in_e;
    c.reached = w.reached;
    c.heavy = w.heavy;
    c.busy = w.busy;
    c.idle = w.idle;
  }
  return c;
}

// First forward level whose path counts may be pushed (levels 0 and 1 have
// counts of 1 and need no count step).
#ifndef BC_FIRST_PUSH_LEVEL
#define BC_FIRST_PUSH_LEVEL 2
#endif
constexpr int kFirstPushLevel = BC_FIRST_PUSH_LEVEL;
#ifndef BC_UNIT_PULL_FACTOR
#define BC_UNIT_PULL_FACTOR 4
#endif
// Level 2 pulls load no counts, so pushing it must save this many times more
// scanned edges than at deeper levels (R-MAT scale 20: +0.7% with 4; the
// directed preferential-attachment graph: equal with 4, -11% with 16).
constexpr unsigned long long kUnitPullFactor = BC_UNIT_PULL_FACTOR;

// Sets the path counts of a level-0 or level-1 entry (one path per source
// bit) in the lane's slots.
template <int W, typename T> __device__ __forceinline__ void unit_counts(T (&s)[2 * W]) {
#pragma unroll
  for (int i = 0; i < 2 * W; ++i) s[i] = 1;
}

// One batch of up to 64*W sources through both sweeps, in the given scope.
// Returns early (leaving the workspace dirty) when the job is in an error
// state.  Warp counters accumulate into cnt (shared, lane 0) and dag (lane).
// CT: storage type of the path counts (uint32_t with promotion of the job to
// 64 bits on the first count that does not fit, or uint64_t).
template <typename DT, int W, bool SQ, typename CT, typename Scope, int S = W>
__device__ __forceinline__ void batch_body(const KParams &p, const Scope sc, int *stage,
                                           WarpCounters &cnt, unsigned long long &dag) {
  const int lane = threadIdx.x & 31;
  const int gwarp = sc.rank() * kWarpsPerBlock + (threadIdx.x >> 5);
  const int nwarps = sc.size() * kWarpsPerBlock;
  const int64_t gtid = (int64_t)sc.rank() * kBlock + threadIdx.x;
  const int64_t nthr = (int64_t)sc.size() * kBlock;
  Ctl *ctl = p.w.ctl;
  const int n = p.g.n;
  const size_t nW = (size_t)n * S; // words of one dense level mask array
  uint64_t *const fr = p.w.fr;
  constexpr int kRow = kK * S;     // sources per state row (of the workspace layout)

  if (read_err(ctl)) return;

  // ---- init: level 0 = the sources (block 0) ------------------------------
  if (sc.rank() == 0) {
    if (threadIdx.x == 0) {
      ctl->tail = 0;
      for (int i = 0; i < kMaxWords; ++i) ctl->ovf[i] = 0;
      ctl->nlevels = 0;
      for (int i = 0; i < 4; ++i) ctl->work[i] = 0;
      p.w.hpack[0] = 0;
      p.w.hpack[1] = 0;
      p.w.qoff[0] = 0;
      p.w.hoff[0] = 0;
      if (p.push_ratio != 0)
        for (int i = 0; i < 4; ++i) p.w.lsum[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x < p.k) {
      const int j = threadIdx.x;
      const int s = __ldg(p.src + j);
      const size_t word = (size_t)s * S + (j >> 6);
      const unsigned long long bit = 1ull << (j & 63);
      atomicOr(reinterpret_cast<unsigned long long *>(p.w.vis + word), bit);
      const uint64_t old = atomicOr(reinterpret_cast<unsigned long long *>(fr + word), bit);
      const bool first = W == 1 ? old == 0 : atomicMax(p.w.claim + s, 1) < 1;
      if (first) {
        const unsigned long long pos = atomicAdd(&ctl->tail, 1ull);
        p.w.qv[pos] = s;
        if (p.push_ratio != 0) {
          atomicAdd(p.w.lsum, (unsigned long long)(__ldg(p.g.in_ptr + s + 1) -
                                                   __ldg(p.g.in_ptr + s)));
          atomicAdd(p.w.lsum + 1, (unsigned long long)(__ldg(p.g.row_ptr + s + 1) -
                                                       __ldg(p.g.row_ptr + s)));
        }
        const int nch = __ldg(p.g.nchunks + s);
        if (nch > 0) {
          const unsigned long long h =
              atomicAdd(&p.w.hpack[0], (1ull << 32) | (unsigned long long)nch);
          p.w.hq_e[h >> 32] = (int64_t)pos;
          p.w.hq_c[h >> 32] = (int64_t)(h & 0xffffffffull);
        }
      }
    }
  }
  if (Scope::kGrid && p.skip_block == sc.rank()) return; // failure-injection hook
  if (!sc.sync(ctl, p.timeout_ns, p.w.qoff + 1)) return;

  // ---- forward sweep -------------------------------------------------------
  LevelView lv;
  lv.lvl = 0;
  lv.lo = 0;
  lv.hi = ldcg(p.w.qoff + 1);
  lv.hoff = 0;
  int64_t lo_m2 = 0; // start of level l-2
  int64_t lo_m1 = 0; // start of level l-1
  int L = 0;
  int step = 0;
  while (true) {
    const int l = lv.lvl;
    uint64_t *Bn = fr + (size_t)((l + 1) & 3) * nW;      // level l+1 (being built)
    const uint64_t *A = fr + (size_t)(l & 3) * nW;       // level l
    const uint64_t *Pm = fr + (size_t)((l + 3) & 3) * nW; // level l-1
    uint64_t *Z = fr + (size_t)((l + 2) & 3) * nW;       // level l-2 (cleared now)
    const unsigned long long hp = ldcg(p.w.hpack + l);
    lv.nheavy = (int64_t)(hp >> 32);
    lv.nhc = (int64_t)(hp & 0xffffffffull);
    lv.hoff_next = lv.hoff + lv.nheavy;
    // direction of this level's path-count step, the same in every block:
    // the degree sums of levels l-1 and l are complete since the last barrier
    // Levels 0 and 1 need no path-count step: in a simple graph a source
    // has one shortest path to itself and one (its edge) to each vertex at
    // depth 1, so their counts are 1 for every source bit.  Level 2 pulls
    // from those counts of 1: its gathers add 1 per set bit and load no row.
    const bool unit_level = l <= 1;
    const bool unit_pull = l == 2;
    bool push = false;
    if (p.push_ratio != 0 && l >= kFirstPushLevel)
      push = p.push_ratio < 0 ||
             (unsigned long long)p.push_ratio * (unit_pull ? kUnitPullFactor : 1) *
                     ldcg(p.w.lsum + 2 * (l - 1) + 1) <
                 ldcg(p.w.lsum + 2 * l);
    if (gtid == 0) {
      p.w.hoff[l] = lv.hoff;
      p.w.hpack[l + 2] = 0;
      if (p.push_ratio != 0) {
        p.w.lsum[2 * (l + 2)] = 0;
        p.w.lsum[2 * (l + 2) + 1] = 0;
      }
      if (push) atomicAdd(p.job_cnt + CNT_PUSH, 1ull);
    }
    zero_ring_ahead(ctl, step, gtid);
    if (l >= 2)
      for (int64_t i = lo_m2 + gtid; i < lo_m1; i += nthr) zero_mask<W, S>(Z, ldcg(p.w.qv + i));

    // push form: the step's first items are the entries of level l-1 (chunks
    // of its heavy entries, then its light entries), pushing their counts
    // along their out-edges; level l's own items then only discover level
    // l+1 and write no counts
    LevelView pv;
    pv.lvl = l - 1;
    pv.lo = lo_m1;
    pv.hi = lv.lo;
    pv.hoff = 0;
    pv.nheavy = 0;
    pv.nhc = 0;
    pv.hoff_next = 0;
    if (push) {
      const unsigned long long hpp = ldcg(p.w.hpack + l - 1);
      pv.hoff = ldcg(p.w.hoff + l - 1);
      pv.nheavy = (int64_t)(hpp >> 32);
      pv.nhc = (int64_t)(hpp & 0xffffffffull);
    }
    const int poff = push ? (int)(pv.nhc + (pv.hi - pv.lo)) : 0;

    unsigned long long *ctr = &ctl->work[step & 3];
    // a step's work items (and the warps' indices into them) are 32-bit:
    // fewer than 2n + 2 x (heavy chunks) < 2^31, which the host checks for
    // every graph a batched job runs on; 64-bit counters here spilled
    const int total = poff + (int)(lv.nhc + (lv.hi - lv.lo));
    trace_step(p, step, l, total, lv.nhc, gtid);
    HeavyCursor hc, hcp;
    int nst = 0; // staged new vertices of this warp
    const int grab = p.grab;
    const int stat = nwarps * grab;
    int base = gwarp * grab;
    const long long t_step = phase_clock();
    while (base < total) {
      const int next = BC_PREFETCH_GROUPS ? (int)next_items(ctr, total, stat, grab, lane) : 0;
      const int end = base + grab < total ? base + grab : total;
      for (int item = base; item < end && item < poff; ++item) {
        // push form: one entry (or one chunk of a heavy entry) of level l-1
        int u, ob, oe;
        if (item < pv.nhc) {
          hcp.seek(p, pv, item, lane);
          u = ldcg(p.w.qv + ldcg(p.w.hq_e + hcp.h));
          const int nch = __ldg(p.g.nchunks + u);
          const int64_t c = item - hcp.first;
          const int rs = __ldg(p.g.row_ptr + u), od = __ldg(p.g.row_ptr + u + 1) - rs;
          ob = rs + (int)(c * od / nch);
          oe = rs + (int)((c + 1) * od / nch);
        } else {
          u = ldcg(p.w.qv + pv.lo + (item - pv.nhc));
          if (__ldg(p.g.nchunks + u) != 0) continue; // heavy: handled as chunks
          ob = __ldg(p.g.row_ptr + u);
          oe = __ldg(p.g.row_ptr + u + 1);
        }
        push_counts<W, CT, S>(p, u, load_mask<W, S>(Pm, u), ob, oe, A, lane, dag);
        if (lane == 0) cnt.out_e += (uint64_t)(oe - ob);
      }
      // level l's own items, numbered from 0
      const int lbase = base > poff ? base - poff : 0;
      const int lend = end > poff ? end - poff : 0;
      for (int item = lbase; item < lend && item < (int)lv.nhc; ++item) {
        // one chunk of a heavy entry
        hc.seek(p, lv, item, lane);
        const int64_t h = hc.h;
        const int64_t e = ldcg(p.w.hq_e + h);
        const int w = ldcg(p.w.qv + e);
        const Mask<W> F = load_mask<W, S>(A, w);
        const int nch = __ldg(p.g.nchunks + w);
        const int64_t c = item - hc.first;
        const int is = __ldg(p.g.in_ptr + w), ie = __ldg(p.g.in_ptr + w + 1);
        const int rs = __ldg(p.g.row_ptr + w), re = __ldg(p.g.row_ptr + w + 1);
        if (push || unit_level) {
          // discovery only, over this chunk's share of the out-edges; the
          // first chunk records the entry (and, at levels 0 and 1, its
          // counts of 1)
          const int od = re - rs;
          const int a = (int)(c * od / nch), b = (int)((c + 1) * od / nch);
          CT s[2 * W] = {};
          unsigned cb = 0;
          fwd_scan<W, CT, S>(p, lv, F, 0, 0, rs + a, rs + b, A, Pm, Bn, stage, nst, lane, s, cb,
                          dag);
          if (unit_level && c == 0) {
            unit_counts<W, CT>(s);
            batch_store_sigma_w<W, CT, CT, S>(p, w, F, s, 0u, lane);
            if (l == 1 && lane == 0) dag += F.popc(); // one DAG edge per source bit
          }
          if (lane == 0) {
            cnt.out_e += (uint64_t)(b - a);
            cnt.heavy++;
            if (c == 0) {
              store_mask<W, S>(p.w.qm, e, F);
              cnt.entries++;
              cnt.reached += F.popc();
            }
          }
          continue;
        }
        const int indeg = ie - is, tot = indeg + (re - rs);
        const int a = (int)(c * tot / nch), b = (int)((c + 1) * tot / nch);
        CT s[2 * W] = {};
        unsigned cb = 0;
        const int ib = is + (a < indeg ? a : indeg), ie2 = is + (b < indeg ? b : indeg);
        const int obg = rs + (a > indeg ? a - indeg : 0);
        const int oen = rs + (b > indeg ? b - indeg : 0);
        fwd_scan<W, CT, S>(p, lv, F, ib, ie2, obg, oen, A, Pm, Bn, stage, nst, lane, s, cb, dag,
                        unit_pull);
        if (lane == 0) {
          cnt.in_e += (uint64_t)((b < indeg ? b : indeg) - (a < indeg ? a : indeg));
          cnt.out_e += (uint64_t)((b > indeg ? b - indeg : 0) - (a > indeg ? a - indeg : 0));
          cnt.heavy++;
        }
        if (nch == 1) {
          // an entry listed with the heavy ones for its size but not split
          // (so it starts early in the step): it stores its counts itself
          batch_store_sigma_w<W, CT, CT, S>(p, w, F, s, cb, lane);
          if (lane == 0) {
            store_mask<W, S>(p.w.qm, e, F);
            cnt.entries++;
            cnt.reached += F.popc();
          }
          continue;
        }
        uint64_t *part = reinterpret_cast<uint64_t *>(p.w.partial) + (size_t)item * kRow;
#pragma unroll
        for (int i = 0; i < 2 * W; ++i) part[32 * i + lane] = s[i];
#pragma unroll
        for (int wi = 0; wi < W; ++wi) {
          const uint64_t ob = (uint64_t)__ballot_sync(kFull, (cb >> (2 * wi)) & 1u) |
                              ((uint64_t)__ballot_sync(kFull, (cb >> (2 * wi + 1)) & 1u) << 32);
          if (lane == 0) p.w.partial_ovf[(size_t)item * S + wi] = ob;
        }
        const unsigned ticket = chunk_ticket(p.w.harrive + h, lane);
        if (ticket == (unsigned)(nch - 1)) {
          const int64_t c0 = hc.first;
          uint64_t t[2 * W] = {};
          unsigned q = 0;
          {
            const uint64_t *pp = reinterpret_cast<const uint64_t *>(p.w.partial);
            for (int64_t cc = c0; cc < c0 + nch; ++cc) {
              uint64_t ow[W];
#pragma unroll
              for (int wi = 0; wi < W; ++wi) ow[wi] = ldcg(p.w.partial_ovf + (size_t)cc * S + wi);
#pragma unroll
              for (int i = 0; i < 2 * W; ++i) {
                bool o = false;
                sat_add(t[i], ldcg(pp + (size_t)cc * kRow + 32 * i + lane), o);
                if (o || ((ow[i >> 1] >> ((i & 1) * 32 + lane)) & 1ull)) q |= 1u << i;
              }
            }
          }
          if (sizeof(CT) == 4) {
            // the chunks' sum must fit the 32-bit storage
            bool big = false;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) big |= F.has(i, lane) && (t[i] >> 32) != 0;
            if (__any_sync(kFull, big)) set_err(ctl, KERR_WIDE);
          }
          batch_store_sigma_w<W, CT, uint64_t, S>(p, w, F, t, q, lane);
          if (lane == 0) {
            p.w.harrive[h] = 0;
            store_mask<W, S>(p.w.qm, e, F);
            cnt.entries++;
            cnt.reached += F.popc();
          }
        }
      }
      if (lend > lv.nhc) {
        using FF = FwdField<W>;
        const int64_t first = lbase > lv.nhc ? lbase : lv.nhc;
        const int64_t e0 = lv.lo + (first - lv.nhc);
        const auto hd = fwd_headers<W, S>(p, A, e0, (int)(lend - first), lane);
        for (int i = 0; i < hd.cnt; ++i) {
          if (hd.field(FF::kNch, i) != 0) continue; // heavy: handled as chunks
          const Mask<W> F = hd.mask(i);
          const int is = (int)hd.field(FF::kIn0, i), ie = (int)hd.field(FF::kIn1, i);
          const int rs = (int)hd.field(FF::kOut0, i), re = (int)hd.field(FF::kOut1, i);
          const int w = (int)hd.field(FF::kId, i);
          CT s[2 * W] = {};
          unsigned cb = 0;
          const bool pull = !unit_level && !push;
          fwd_scan<W, CT, S>(p, lv, F, pull ? is : 0, pull ? ie : 0, rs, re, A, Pm, Bn, stage, nst,
                          lane, s, cb, dag, unit_pull);
          if (unit_level) {
            unit_counts<W, CT>(s);
            if (l == 1 && lane == 0) dag += F.popc(); // one DAG edge per source bit
          }
          if (!push) batch_store_sigma_w<W, CT, CT, S>(p, w, F, s, cb, lane);
          if (lane == 0) {
            store_mask<W, S>(p.w.qm, e0 + i, F);
            cnt.entries++;
            cnt.reached += F.popc();
            cnt.in_e += (uint64_t)(pull ? ie - is : 0);
            cnt.out_e += (uint64_t)(re - rs);
          }
        }
      }
      base = BC_PREFETCH_GROUPS ? next : (int)next_items(ctr, total, stat, grab, lane);
    }
    __syncwarp();
    stage_flush(p, lv, stage, nst, lane);
    const long long t_done = phase_clock();
    if (!sc.sync(ctl, p.timeout_ns, p.w.qoff + l + 2)) return;
    if (lane == 0) {
      cnt.busy += (unsigned long long)(t_done - t_step);
      cnt.idle += (unsigned long long)(phase_clock() - t_done);
    }
    ++step;
    const int64_t nh = ldcg(p.w.qoff + l + 2);
    if (nh == lv.hi) {
      L = l + 1;
      break;
    }
    lo_m2 = lo_m1;
    lo_m1 = lv.lo;
    lv.lo = lv.hi;
    lv.hi = nh;
    lv.hoff = lv.hoff_next;
    lv.lvl = l + 1;
  }

  if (gtid == 0) {
    ctl->nlevels = L;
    atomicMax(p.job_cnt + CNT_MAXLEV, (unsigned long long)L);
    atomicAdd(p.job_cnt + CNT_LEVELS, (unsigned long long)L);
    for (int wi = 0; wi < W; ++wi) {
      const uint64_t ob = ldcg(&ctl->ovf[wi]);
      for (int j = 64 * wi; j < p.k && j < 64 * (wi + 1); ++j)
        if ((ob >> (j & 63)) & 1ull) p.ovf_flags[p.src_base + j] = 1;
    }
  }

  // ---- backward sweep ------------------------------------------------------
  for (int l = L - 1; l >= 0; --l) {
    const uint64_t *Dn = fr + (size_t)((l + 1) & 3) * nW; // level l+1 masks
    uint64_t *Wn = l > 0 ? fr + (size_t)(l & 3) * nW : nullptr; // level l masks for step l-1
    uint64_t *Z = fr + (size_t)((l + 2) & 3) * nW;        // level l+2 (cleared now)
    LevelView bl;
    bl.lvl = l;
    bl.lo = ldcg(p.w.qoff + l);
    bl.hi = ldcg(p.w.qoff + l + 1);
    const unsigned long long hp = ldcg(p.w.hpack + l);
    bl.nheavy = (int64_t)(hp >> 32);
    bl.nhc = (int64_t)(hp & 0xffffffffull);
    bl.hoff = ldcg(p.w.hoff + l);
    bl.hoff_next = 0;
    zero_ring_ahead(ctl, step, gtid);
    if (l + 2 <= L - 1) {
      const int64_t zlo = ldcg(p.w.qoff + l + 2), zhi = ldcg(p.w.qoff + l + 3);
      for (int64_t i = zlo + gtid; i < zhi; i += nthr) zero_mask<W, S>(Z, ldcg(p.w.qv + i));
    }
    // the deepest level has no successors; at level 0 every source bit is
    // the vertex itself, whose own dependency no BC term uses (only debug
    // exports report it)
    const bool gather = l < L - 1 && (l > 0 || p.dbg_d != nullptr);
    unsigned long long *ctr = &ctl->work[step & 3];
    const int total = (int)(bl.nhc + (bl.hi - bl.lo));
    trace_step(p, step, -1 - l, total, bl.nhc, gtid);
    HeavyCursor hc;
    const int grab = p.grab;
    const int stat = nwarps * grab;
    int base = gwarp * grab;
    const long long t_step = phase_clock();
    while (base < total) {
      const int next = BC_PREFETCH_GROUPS ? (int)next_items(ctr, total, stat, grab, lane) : 0;
      const int end = base + grab < total ? base + grab : total;
      for (int item = base; item < end && item < (int)bl.nhc; ++item) {
        hc.seek(p, bl, item, lane);
        const int64_t h = hc.h;
        const int64_t e = ldcg(p.w.hq_e + h);
        const int v = ldcg(p.w.qv + e);
        const Mask<W> F = load_mask<W, S>(p.w.qm, e);
        const int nch = __ldg(p.g.nchunks + v);
        const int64_t c = item - hc.first;
        const int rs = __ldg(p.g.row_ptr + v), re = __ldg(p.g.row_ptr + v + 1);
        const int od = re - rs;
        const int a = (int)(c * od / nch), b = (int)((c + 1) * od / nch);
        DT acc[2 * W] = {};
        if (gather) batch_pull_delta_w<W, DT, S>(p, F, rs + a, rs + b, Dn, lane, acc);
        if (lane == 0) {
          cnt.out_e += (uint64_t)(gather ? b - a : 0);
          cnt.heavy++;
        }
        if (nch == 1) { // not split: the entry closes itself
          const EntryOwn<W, CT, S> own(p, v, F, lane);
          batch_finish<DT, W, SQ, CT, S>(p, l, v, F, acc, own.sg, own.bcv, Wn, lane);
          continue;
        }
        DT *part = reinterpret_cast<DT *>(p.w.partial) + (size_t)item * kRow;
#pragma unroll
        for (int i = 0; i < 2 * W; ++i) part[32 * i + lane] = acc[i];
        const unsigned ticket = chunk_ticket(p.w.harrive + h, lane);
        if (ticket == (unsigned)(nch - 1)) {
          const int64_t c0 = hc.first;
          const DT *pp = reinterpret_cast<const DT *>(p.w.partial);
          DT t[2 * W] = {};
          for (int64_t cc = c0; cc < c0 + nch; ++cc)
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) t[i] += ldcg(pp + (size_t)cc * kRow + 32 * i + lane);
          const EntryOwn<W, CT, S> own(p, v, F, lane);
          batch_finish<DT, W, SQ, CT, S>(p, l, v, F, t, own.sg, own.bcv, Wn, lane);
          if (lane == 0) p.w.harrive[h] = 0;
        }
      }
      if (end > bl.nhc) {
        using BF = BwdField<W>;
        const int64_t first = base > bl.nhc ? base : bl.nhc;
        const int64_t e0 = bl.lo + (first - bl.nhc);
        const auto hd = bwd_headers<W, S>(p, e0, (int)(end - first), lane);
        for (int i = 0; i < hd.cnt; ++i) {
          if (hd.field(BF::kNch, i) != 0) continue;
          const Mask<W> F = hd.mask(i);
          const int rs = (int)hd.field(BF::kOut0, i), re = (int)hd.field(BF::kOut1, i);
          const int v = (int)hd.field(BF::kId, i);
          DT acc[2 * W] = {};
          if constexpr (W <= BC_OWN_EARLY_MAX_W) {
            // own counts loaded ahead of the successor scan (overlapping it)
            const EntryOwn<W, CT, S> own(p, v, F, lane);
            if (gather) batch_pull_delta_w<W, DT, S>(p, F, rs, re, Dn, lane, acc);
            batch_finish<DT, W, SQ, CT, S>(p, l, v, F, acc, own.sg, own.bcv, Wn, lane);
          } else {
            // widest masks: loaded after it, which keeps 4W registers free
            if (gather) batch_pull_delta_w<W, DT, S>(p, F, rs, re, Dn, lane, acc);
            const EntryOwn<W, CT, S> own(p, v, F, lane);
            batch_finish<DT, W, SQ, CT, S>(p, l, v, F, acc, own.sg, own.bcv, Wn, lane);
          }
          if (gather && lane == 0) cnt.out_e += (uint64_t)(re - rs);
        }
      }
      base = BC_PREFETCH_GROUPS ? next : (int)next_items(ctr, total, stat, grab, lane);
    }
    const long long t_done = phase_clock();
    if (!sc.sync(ctl, p.timeout_ns)) return;
    if (lane == 0) {
      cnt.busy += (unsigned long long)(t_done - t_step);
      cnt.idle += (unsigned long long)(phase_clock() - t_done);
    }
    ++step;
  }

  trace_step(p, step, 1 << 20, 0, 0, gtid); // end marker

  // ---- leave the workspace clean for the next batch ------------------------
  {
    const int64_t q1 = ldcg(p.w.qoff + 1);
    const int64_t q2 = L >= 2 ? ldcg(p.w.qoff + 2) : q1;
    for (int64_t i = gtid; i < q1; i += nthr) zero_mask<W, S>(fr, ldcg(p.w.qv + i));
    for (int64_t i = q1 + gtid; i < q2; i += nthr) zero_mask<W, S>(fr + nW, ldcg(p.w.qv + i));
  }
}

template <typename DT, int W, bool SQ, typename CT, int S = W>
__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) batch_kernel(const KParams p) {
  __shared__ int s_stage[kWarpsPerBlock][kStage]; // warp-private new-vertex stage
  __shared__ WarpCounters s_cnt[kWarpsPerBlock];
  const int lane = threadIdx.x & 31;
  WarpCounters &cnt = s_cnt[threadIdx.x >> 5];
  zero_counters(cnt, lane);
  unsigned long long dag = 0;
  batch_body<DT, W, SQ, CT, GridScope, S>(p, GridScope(), s_stage[threadIdx.x >> 5], cnt, dag);
  __syncwarp();
  flush_counters(p.job_cnt, to_counters(cnt, dag, lane), lane);
}

// A job's batches in concurrent groups (MultiParams): fewer SMs per batch
// make each step's work per warp larger against the fixed costs of a step
// (the barrier and the last items' tail), which dominate the small steps of
// small graphs and of deep, narrow traversals.  Every group adds its batches
// in order into its own BC partial vector; the host sums the vectors in
// group order, so results repeat bit for bit.
template <typename DT, int W, bool SQ, typename CT>
__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) multi_batch_kernel(const MultiParams mp) {
  __shared__ int s_stage[kWarpsPerBlock][kStage];
  __shared__ WarpCounters s_cnt[kWarpsPerBlock];
  __shared__ KParams sp;
  const int lane = threadIdx.x & 31;
  WarpCounters &cnt = s_cnt[threadIdx.x >> 5];
  zero_counters(cnt, lane);
  unsigned long long dag = 0;
  const GroupScope sc{(int)blockIdx.x / mp.gsize, mp.gsize};
  const int64_t nbatch = (mp.k - mp.first + mp.kb - 1) / mp.kb;
  if (threadIdx.x == 0) {
    sp = mp.base;
    sp.w = mp.works[sc.g];
    sp.bc = mp.parts + (size_t)sc.g * (size_t)mp.base.g.n;
    sp.trace = nullptr;
    sp.skip_block = -1;
  }
  for (int64_t b = sc.g; b < nbatch; b += mp.groups) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t s0 = mp.first + b * mp.kb;
      sp.src = mp.base.src + s0;
      sp.k = (int32_t)(mp.k - s0 < mp.kb ? mp.k - s0 : mp.kb);
      sp.src_base = s0;
    }
    __syncthreads();
    batch_body<DT, W, SQ, CT>(sp, sc, s_stage[threadIdx.x >> 5], cnt, dag);
    // the next batch's set-up must not meet this one's final clean-up
    if (!sc.sync(sp.w.ctl, sp.timeout_ns)) break;
  }
  __syncwarp();
  flush_counters(mp.base.job_cnt, to_counters(cnt, dag, lane), lane);
}

// Clears what a batch stopped in its forward sweep may leave behind in a
// block's workspace and must be clean at a batch's start: visited and level
// masks, first-toucher claims, chunk tickets and the error code.  (Path
// counts and coefficients are only read where this batch wrote them.)
__device__ void block_reset_workspace(const Work &w, int n) {
  const size_t words = (size_t)n * (size_t)w.words;
  for (size_t i = threadIdx.x; i < words; i += blockDim.x) w.vis[i] = 0;
  for (size_t i = threadIdx.x; i < 4 * words; i += blockDim.x) w.fr[i] = 0;
  if (w.claim)
    for (int i = threadIdx.x; i < n; i += blockDim.x) w.claim[i] = 0;
  for (int64_t i = threadIdx.x; i < w.hcap; i += blockDim.x) w.harrive[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) w.ctl->err = KERR_NONE;
  __syncthreads();
}

// One batch of the many-graph launch with `words` mask words and path-count
// rows of CT.
template <typename DT, typename CT>
__device__ __forceinline__ void many_batch(const KParams &p, int words, int *stage,
                                           WarpCounters &cnt, unsigned long long &dag) {
  if (words == 4) batch_body<DT, 4, false, CT>(p, CtaScope(), stage, cnt, dag);
  else if (words == 2) batch_body<DT, 2, false, CT>(p, CtaScope(), stage, cnt, dag);
  else batch_body<DT, 1, false, CT>(p, CtaScope(), stage, cnt, dag);
}

// Exact BC of many small graphs in one launch: each thread block takes the
// next graph from a shared counter (largest work first) and runs all of that
// graph's source batches itself, with CTA barriers between levels, so every
// graph's BC is written by one block without atomics.  Each graph gets its
// own batch width (auto_words of its vertex count, up to mp.max_words) and
// starts with 32-bit path-count rows unless mp.counts64.  A batch that
// cannot finish in its configuration stops in its forward sweep, before any
// BC is written, and is run again: after a queue overrun of a wide batch
// the graph's remaining sources continue 64 per batch, after a count of
// 2^32 or more with 64-bit rows.  Sources without out-edges, last in the
// grouped order, are not run (their dependencies are all zero).
template <typename DT>
__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) many_kernel(const ManyParams mp) {
  __shared__ int s_stage[kWarpsPerBlock][kStage];
  __shared__ WarpCounters s_cnt[kWarpsPerBlock];
  __shared__ int s_item;
  const int lane = threadIdx.x & 31;
  WarpCounters &cnt = s_cnt[threadIdx.x >> 5];
  zero_counters(cnt, lane);
  unsigned long long dag = 0;
  KParams p = mp.base;
  p.w = mp.works[blockIdx.x];
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(mp.next, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= mp.count || read_err(p.w.ctl)) break;
    const int gi = __ldg(mp.order + it);
    p.g = mp.graphs[gi];
    const int64_t off = __ldg(mp.out_off + gi);
    const int nt = __ldg(mp.traverse + gi);
    p.bc = mp.out + off;
    int words = mp.max_words > 1 ? auto_words(p.g.n, mp.max_words) : 1;
    bool wide = mp.counts64 != 0;
    for (int b0 = 0; b0 < nt;) {
      const int kb = words > 1 ? kK * words : mp.kb;
      p.src = (mp.grouped && p.g.order ? p.g.order : mp.iota) + b0;
      p.k = nt - b0 < kb ? nt - b0 : kb;
      p.src_base = off + b0;
      if (wide) many_batch<DT, uint64_t>(p, words, s_stage[threadIdx.x >> 5], cnt, dag);
      else many_batch<DT, uint32_t>(p, words, s_stage[threadIdx.x >> 5], cnt, dag);
      __syncthreads();
      const int e = read_err(p.w.ctl);
      if ((e == KERR_QUEUE || e == KERR_HEAVY) && words > 1) {
        block_reset_workspace(p.w, p.g.n);
        words = 1; // redo these sources 64 per batch
        continue;
      }
      if (e == KERR_WIDE && !wide) {
        block_reset_workspace(p.w, p.g.n);
        wide = true; // redo these sources with 64-bit counts
        continue;
      }
      if (e) break;
      b0 += p.k;
    }
  }
  __syncwarp();
  flush_counters(p.job_cnt, to_counters(cnt, dag, lane), lane);
}

} // namespace
} // namespace bcgpu
