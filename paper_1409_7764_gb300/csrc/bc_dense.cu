// Dense-level batched kernel: up to 64 sources per persistent launch, with
// the frontier of every BFS level kept as a dense array of u64 masks.
//
// Same method as the queue kernel in bc_kernels.cu (Brandes' forward BFS with
// path counts, then the reverse dependency sweep, paper Section I), but the
// frontier of level l is the dense array lm[l][v] (bit j = vertex v is at
// depth l from source j) instead of a queue:
//   - discovery ORs new bits into lm[l+1][x] with a reduction that returns
//     nothing, so no warp waits on an atomic and no queue is built;
//   - the backward sweep reads lm[l] for its entries and lm[l+1] for the
//     successor test, so no per-entry record is kept between the sweeps;
//   - a step scans all n masks of its level in groups of kGroup = 8 vertices;
//     a warp processes the active light vertices of a group together, with
//     their edges flattened across the 32 lanes (one round of loads covers
//     several vertices) and their per-source sums held in shared memory
//     (lane j owns sources j and j+32, so no two lanes touch one slot);
//   - high-degree vertices are cut into kChunk-edge chunks listed once per
//     graph; partial sums meet in scratch and the last chunk to arrive reduces
//     them in chunk order (deterministic);
//   - each CTA owns a fixed strided share of the step's work items and its
//     warps take items from a shared-memory counter (no global counter).
// Levels beyond the mask array's capacity (dmax) stop the launch with
// KERR_LEVELS before any BC is written; the host then reruns the job with the
// queue kernel.
#include "bc_device.cuh"

namespace bcgpu {
namespace {

constexpr int kAcc = kGroup * kK; // accumulator slots per warp

struct DenseSmem {
  unsigned long long acc[kWarpsPerBlock][kAcc]; // per-warp [kGroup][64] sums (u64 or DT view)
  double red[kWarpsPerBlock][kGroup][kWarp];    // per-warp BC contributions before reduction
  unsigned long long ovf[kWarpsPerBlock][kGroup]; // per-warp carry bits of each entry's counts
  unsigned long long next;                      // CTA-local item counter
};

// Exclusive prefix over lanes 0..kGroup-1 (other lanes: don't care) and the
// group total, broadcast to all lanes.
__device__ __forceinline__ int group_excl_scan(int x, int lane, int &total) {
  int inc = x;
#pragma unroll
  for (int off = 1; off < kGroup; off <<= 1) {
    const int t = __shfl_up_sync(kFull, inc, off, kGroup);
    if ((lane & (kGroup - 1)) >= off) inc += t;
  }
  total = __shfl_sync(kFull, inc, kGroup - 1);
  return inc - x;
}

// Owner entry of flattened edge t: the largest i with start[i] <= t.
__device__ __forceinline__ int group_owner(int start, int t) {
  int i = 0;
#pragma unroll
  for (int k = 1; k < kGroup; ++k)
    if (__shfl_sync(kFull, start, k) <= t) i = k;
  return i;
}

// Per-step view of the level's heavy-vertex list (vertices with chunks):
// entries [hoff, hoff + nheavy) of hq_e (vertex ids) / hq_c (first chunk of
// the vertex within the level); nhc chunks in total; the next level's list
// starts at hoff_next.
struct HeavyLevel {
  int lvl;
  int64_t hoff, nheavy, nhc, hoff_next;
};

// Records heavy vertex x (nch chunks) as active at level `lvl` (called once,
// by the discovery that first set a bit of x at that level).
__device__ __forceinline__ void heavy_enqueue(const KParams &p, int lvl, int64_t hoff_lvl, int x,
                                              int nch) {
  const unsigned long long h =
      atomicAdd(&p.w.hpack[lvl], (1ull << 32) | (unsigned long long)nch);
  const int64_t hidx = hoff_lvl + (int64_t)(h >> 32);
  const int64_t cpre = (int64_t)(h & 0xffffffffull);
  if (hidx >= p.w.hcap) {
    set_err(p.w.ctl, KERR_HEAVY);
    return;
  }
  if (cpre + nch > p.w.chunk_cap) {
    set_err(p.w.ctl, KERR_CHUNKS);
    return;
  }
  p.w.hq_e[hidx] = x;
  p.w.hq_c[hidx] = cpre;
}

// New bits m for vertex x at the next level: a fire-and-forget OR for a light
// vertex; for a heavy one the OR's old value tells whether this is its first
// bit at that level, and the first discoverer lists it.
__device__ __forceinline__ void push_bits(const KParams &p, const HeavyLevel &hl, uint64_t *Bn,
                                          int x, int ncx, uint64_t m) {
  if (!Bn) {
    set_err(p.w.ctl, KERR_LEVELS);
    return;
  }
  if (ncx == 0) {
    atomicOr(reinterpret_cast<unsigned long long *>(Bn + x), m);
  } else {
    const uint64_t old = atomicOr(reinterpret_cast<unsigned long long *>(Bn + x), m);
    if (old == 0) heavy_enqueue(p, hl.lvl + 1, hl.hoff_next, x, ncx);
  }
}

// Discovery push of one frontier vertex over out-edges [eb, ee).
__device__ __forceinline__ bool dense_discover(const KParams &p, const HeavyLevel &hl, uint64_t F,
                                               int64_t eb, int64_t ee, const uint64_t *A,
                                               uint64_t *Bn, int lane) {
  bool any = false;
  for (int64_t base = eb; base < ee; base += kWarp) {
    const int64_t e = base + lane;
    if (e < ee) {
      const int x = __ldg(p.g.col_idx + e);
      const int ncx = __ldg(p.g.nchunks + x);
      const uint64_t m = F & ~(ldcg(p.w.vis + x) | ldcg(A + x));
      if (m) {
        push_bits(p, hl, Bn, x, ncx, m);
        any = true;
      }
    }
  }
  return any;
}

// Closes one backward entry (vertex v, mask F) from the lane's successor sums:
// dependencies and coefficients (path counts need no reset: they are only
// read where the same batch wrote them); returns the lane's BC contribution.
template <typename DT>
__device__ __forceinline__ double dense_close(const KParams &p, int lvl, int v, uint64_t F, DT a0,
                                              DT a1, int s_lo, int s_hi, int lane) {
  const uint64_t *srow = p.w.sigma + (size_t)v * kK;
  DT *crow = reinterpret_cast<DT *>(p.w.cdep) + (size_t)v * kK;
  double contrib = 0.0;
  const int n = p.g.n;
  if ((F >> lane) & 1ull) {
    const uint64_t sg = ldcg(srow + lane);
    const DT sf = u64_to<DT>(sg);
    const DT dl = sf * a0;
    crow[lane] = (DT(1) + dl) / sf;
    if (s_lo != v) contrib += (double)dl;
    if (p.dbg_d) {
      const size_t o = (size_t)lane * n + v;
      p.dbg_d[o] = lvl;
      p.dbg_sigma[o] = sg;
      p.dbg_delta[o] = (double)dl;
    }
  }
  if ((F >> (lane + 32)) & 1ull) {
    const uint64_t sg = ldcg(srow + 32 + lane);
    const DT sf = u64_to<DT>(sg);
    const DT dl = sf * a1;
    crow[32 + lane] = (DT(1) + dl) / sf;
    if (s_hi != v) contrib += (double)dl;
    if (p.dbg_d) {
      const size_t o = (size_t)(lane + 32) * n + v;
      p.dbg_d[o] = lvl;
      p.dbg_sigma[o] = sg;
      p.dbg_delta[o] = (double)dl;
    }
  }
  return contrib;
}

// ---- forward: one group of kGroup light vertices ------------------------------
template <typename DT>
__device__ void fwd_group(const KParams &p, const HeavyLevel &hl, int64_t v0, const uint64_t *A,
                          uint64_t *Bn, const uint64_t *Pm, unsigned long long *acc,
                          unsigned long long *govf, int lane, Counters &cnt, bool &any_new) {
  const int l = hl.lvl;
  const int n = p.g.n;
  const int gi = lane & (kGroup - 1);
  const int64_t vv = v0 + gi;
  uint64_t F = 0;
  if (lane < kGroup && vv < n) {
    const uint64_t fm = ldcg(A + vv);
    const int nc = __ldg(p.g.nchunks + vv);
    F = nc ? 0ull : fm; // heavy vertices run as chunks
  }
  const unsigned amask = __ballot_sync(kFull, F != 0);
  if (!amask) return;
  const int f = lane >> 3;
  int hv = 0;
  if ((amask >> gi) & 1u) {
    const int64_t vi = v0 + gi;
    hv = f == 0 ? __ldg(p.g.in_ptr + vi)
                : f == 1 ? __ldg(p.g.in_ptr + vi + 1)
                         : f == 2 ? __ldg(p.g.row_ptr + vi) : __ldg(p.g.row_ptr + vi + 1);
  }
  const int is = __shfl_sync(kFull, hv, gi), ie = __shfl_sync(kFull, hv, 8 + gi);
  const int rs = __shfl_sync(kFull, hv, 16 + gi), re = __shfl_sync(kFull, hv, 24 + gi);
  const bool act = lane < kGroup && ((amask >> lane) & 1u);
  int Tin = 0, Tout = 0;
  const int din = (act && l > 0) ? ie - is : 0;
  const int dout = act ? re - rs : 0;
  const int pin = group_excl_scan(din, lane, Tin);
  const int pout = group_excl_scan(dout, lane, Tout);

  // owners record the level in their visited masks
  if (act) p.w.vis[vv] = ldcg(p.w.vis + vv) | F;

  // path counts: pull over the flattened in-edges of all active vertices;
  // lanes take edges and add into their entry's shared row
  if (l > 0) {
#pragma unroll
    for (int i = 0; i < kGroup; ++i)
      if ((amask >> i) & 1u) {
        acc[i * kK + lane] = 0;
        acc[i * kK + 32 + lane] = 0;
      }
    if (lane < kGroup) govf[lane] = 0;
    __syncwarp();
    unsigned long long nd = 0;
    for (int base = 0; base < Tin; base += kWarp) {
      const int t = base + lane;
      const int i = group_owner(pin, t);
      const int isi = __shfl_sync(kFull, is, i);
      const int pini = __shfl_sync(kFull, pin, i);
      const uint64_t Fi = __shfl_sync(kFull, F, i);
      if (t < Tin) {
        const int u = __ldg(p.g.in_idx + isi + (t - pini));
        const uint64_t P = ldcg(Pm + u) & Fi;
        nd += __popcll(P);
        uint64_t ol = 0;
        gather_counts(p.w.sigma + (size_t)u * kK, P, acc + i * kK, ol);
        if (ol) atomicOr(govf + i, (unsigned long long)ol);
      }
    }
    nd = warp_sum_u64(nd);
    if (lane == 0) cnt.dag += nd;
    __syncwarp();
  }
  // store the path counts (level 0: the sources, count 1; saturated on carry)
#pragma unroll
  for (int i = 0; i < kGroup; ++i) {
    if (!((amask >> i) & 1u)) continue;
    const uint64_t Fi = __shfl_sync(kFull, F, i);
    const uint64_t oi = l > 0 ? govf[i] & Fi : 0ull;
    uint64_t *row = p.w.sigma + (size_t)(v0 + i) * kK;
    if ((Fi >> lane) & 1ull)
      row[lane] = l == 0 ? 1ull : (((oi >> lane) & 1ull) ? ~0ull : (uint64_t)acc[i * kK + lane]);
    if ((Fi >> (lane + 32)) & 1ull)
      row[32 + lane] = l == 0 ? 1ull
                              : (((oi >> (lane + 32)) & 1ull) ? ~0ull
                                                              : (uint64_t)acc[i * kK + 32 + lane]);
    if (oi && lane == 0) atomicOr(&p.w.ctl->ovf[0], (unsigned long long)oi);
  }
  __syncwarp();
  // discovery: flattened out-edges of all active vertices
  bool any = false;
  for (int base = 0; base < Tout; base += kWarp) {
    const int t = base + lane;
    const int i = group_owner(pout, t);
    const int rsi = __shfl_sync(kFull, rs, i);
    const int pouti = __shfl_sync(kFull, pout, i);
    const uint64_t Fi = __shfl_sync(kFull, F, i);
    if (t < Tout) {
      const int x = __ldg(p.g.col_idx + rsi + (t - pouti));
      const int ncx = __ldg(p.g.nchunks + x);
      const uint64_t m = Fi & ~(ldcg(p.w.vis + x) | ldcg(A + x));
      if (m) {
        push_bits(p, hl, Bn, x, ncx, m);
        any = true;
      }
    }
  }
  any_new |= any;
  if (act) {
    cnt.entries++;
    cnt.reached += __popcll(F);
  }
  if (lane == 0) {
    cnt.in_e += (unsigned long long)Tin;
    cnt.out_e += (unsigned long long)Tout;
  }
}

// ---- backward: one group of kGroup light vertices -------------------------------
template <typename DT>
__device__ void bwd_group(const KParams &p, int l, int64_t v0, const uint64_t *A,
                          const uint64_t *Dn, unsigned long long *accraw, double *red, int s_lo,
                          int s_hi, int lane, Counters &cnt) {
  const int n = p.g.n;
  const int gi = lane & (kGroup - 1);
  const int64_t vv = v0 + gi;
  uint64_t F = 0;
  if (lane < kGroup && vv < n) {
    const uint64_t fm = ldcg(A + vv);
    const int nc = __ldg(p.g.nchunks + vv);
    F = nc ? 0ull : fm;
  }
  const unsigned amask = __ballot_sync(kFull, F != 0);
  if (!amask) return;
  DT *acc = reinterpret_cast<DT *>(accraw);
  int rs = 0, re = 0, Tout = 0;
  if (Dn) {
    const int f = lane >> 3;
    int hv = 0;
    if (f < 2 && ((amask >> gi) & 1u))
      hv = f == 0 ? __ldg(p.g.row_ptr + v0 + gi) : __ldg(p.g.row_ptr + v0 + gi + 1);
    rs = __shfl_sync(kFull, hv, gi);
    re = __shfl_sync(kFull, hv, 8 + gi);
  }
  const bool act = lane < kGroup && ((amask >> lane) & 1u);
  const int dout = (act && Dn) ? re - rs : 0;
  const int pout = group_excl_scan(dout, lane, Tout);
#pragma unroll
  for (int i = 0; i < kGroup; ++i)
    if ((amask >> i) & 1u) {
      acc[i * kK + lane] = DT(0);
      acc[i * kK + 32 + lane] = DT(0);
    }
  __syncwarp();
  // successor sums over the flattened out-edges; lanes take edges and add the
  // successors' coefficients into their entry's shared row
  const DT *cdep = reinterpret_cast<const DT *>(p.w.cdep);
  for (int base = 0; base < Tout; base += kWarp) {
    const int t = base + lane;
    const int i = group_owner(pout, t);
    const int rsi = __shfl_sync(kFull, rs, i);
    const int pouti = __shfl_sync(kFull, pout, i);
    const uint64_t Fi = __shfl_sync(kFull, F, i);
    if (t < Tout) {
      const int x = __ldg(p.g.col_idx + rsi + (t - pouti));
      const uint64_t S = ldcg(Dn + x) & Fi;
      gather_coeffs<DT>(cdep + (size_t)x * kK, S, acc + i * kK);
    }
  }
  __syncwarp();
  // close every active entry; reduce the BC contributions in lane order
#pragma unroll
  for (int i = 0; i < kGroup; ++i) {
    double c = 0.0;
    if ((amask >> i) & 1u) {
      const uint64_t Fi = __shfl_sync(kFull, F, i);
      c = dense_close<DT>(p, l, (int)(v0 + i), Fi, acc[i * kK + lane], acc[i * kK + 32 + lane],
                          s_lo, s_hi, lane);
    }
    red[i * kWarp + lane] = c;
  }
  __syncwarp();
  if (act) {
    double sum = 0.0;
    for (int j = 0; j < kWarp; ++j) sum += red[lane * kWarp + j];
    if (sum != 0.0) p.bc[vv] = ldcg(p.bc + vv) + sum;
    p.w.vis[vv] = 0;
    cnt.entries++;
  }
  __syncwarp();
  if (lane == 0) cnt.out_e += (unsigned long long)Tout;
}

// ---- heavy chunks -------------------------------------------------------------------

// The heavy entry owning chunk `item` of the level and that chunk's edge share.
struct ChunkRef {
  int64_t h;     // heavy entry
  int v;         // vertex
  int nch;       // chunks of v
  int64_t first; // first chunk of v within the level
  int64_t ci;    // this chunk's index within v
};

__device__ __forceinline__ ChunkRef chunk_ref(const KParams &p, const HeavyLevel &hl,
                                              int64_t item, int lane) {
  ChunkRef r;
  r.h = warp_find_heavy(p.w.hq_c, hl.hoff, hl.nheavy, item, lane);
  r.v = (int)ldcg(p.w.hq_e + r.h);
  r.first = ldcg(p.w.hq_c + r.h);
  r.ci = item - r.first;
  r.nch = __ldg(p.g.nchunks + r.v);
  return r;
}

// Forward work of chunk `item` of the level.
template <typename DT>
__device__ void fwd_chunk(const KParams &p, const HeavyLevel &hl, int64_t item,
                          const uint64_t *A, uint64_t *Bn, const uint64_t *Pm,
                          unsigned long long *wacc, int lane, Counters &cnt, bool &any_new) {
  const int l = hl.lvl;
  const ChunkRef r = chunk_ref(p, hl, item, lane);
  const int v = r.v, nch = r.nch;
  const uint64_t F = ldcg(A + v);
  const int64_t is = __ldg(p.g.in_ptr + v), ie = __ldg(p.g.in_ptr + v + 1);
  const int64_t rs = __ldg(p.g.row_ptr + v), re = __ldg(p.g.row_ptr + v + 1);
  const int64_t indeg = ie - is, tot = indeg + (re - rs);
  const int64_t a = r.ci * tot / nch, b = (r.ci + 1) * tot / nch;
  uint64_t s0 = 0, s1 = 0;
  bool o0 = false, o1 = false;
  if (l > 0 && a < indeg)
    batch_pull_sigma(p, F, is + a, is + (b < indeg ? b : indeg), Pm, lane, wacc, s0, s1, o0, o1,
                     cnt.dag);
  if (b > indeg)
    any_new |= dense_discover(p, hl, F, rs + (a > indeg ? a - indeg : 0), rs + (b - indeg), A,
                              Bn, lane);
  if (lane == 0) {
    cnt.in_e += (uint64_t)(l > 0 ? (b < indeg ? b : indeg) - (a < indeg ? a : indeg) : 0);
    cnt.out_e += (uint64_t)((b > indeg ? b - indeg : 0) - (a > indeg ? a - indeg : 0));
    cnt.heavy++;
  }
  uint64_t *part = reinterpret_cast<uint64_t *>(p.w.partial) + (size_t)item * kK;
  part[lane] = s0;
  part[32 + lane] = s1;
  const uint64_t ob = (uint64_t)__ballot_sync(kFull, o0) | ((uint64_t)__ballot_sync(kFull, o1) << 32);
  if (lane == 0) p.w.partial_ovf[item] = ob;
  const unsigned ticket = chunk_ticket(p.w.harrive + r.h, lane);
  if (ticket != (unsigned)(nch - 1)) return;
  // last chunk of v: reduce the partials in chunk order
  uint64_t t0 = 0, t1 = 0;
  bool q0 = false, q1 = false;
  uint64_t ovb = 0;
  if (l == 0) {
    t0 = 1;
    t1 = 1;
  } else {
    const uint64_t *pp = reinterpret_cast<const uint64_t *>(p.w.partial);
#pragma unroll 4
    for (int64_t cc = r.first; cc < r.first + nch; ++cc) {
      sat_add(t0, ldcg(pp + (size_t)cc * kK + lane), q0);
      sat_add(t1, ldcg(pp + (size_t)cc * kK + 32 + lane), q1);
      ovb |= ldcg(p.w.partial_ovf + cc);
    }
  }
  batch_store_sigma(p, v, F, t0, t1, q0 || ((ovb >> lane) & 1ull),
                    q1 || ((ovb >> (lane + 32)) & 1ull), lane);
  if (lane == 0) {
    p.w.harrive[r.h] = 0;
    p.w.vis[v] = ldcg(p.w.vis + v) | F;
    cnt.entries++;
    cnt.reached += __popcll(F);
  }
}

// Backward work of chunk `item` of the level.
template <typename DT>
__device__ void bwd_chunk(const KParams &p, const HeavyLevel &hl, int64_t item,
                          const uint64_t *A, const uint64_t *Dn, unsigned long long *wacc,
                          double *red, int s_lo, int s_hi, int lane, Counters &cnt) {
  const int l = hl.lvl;
  const ChunkRef r = chunk_ref(p, hl, item, lane);
  const int v = r.v, nch = r.nch;
  const uint64_t F = ldcg(A + v);
  const int64_t rs = __ldg(p.g.row_ptr + v), re = __ldg(p.g.row_ptr + v + 1);
  const int64_t od = re - rs;
  const int64_t a = r.ci * od / nch, b = (r.ci + 1) * od / nch;
  (void)wacc;
  DT acc[2] = {DT(0), DT(0)};
  if (Dn) {
    Mask<1> FM;
    FM.w[0] = F;
    batch_pull_delta_w<1, DT>(p, FM, rs + a, rs + b, Dn, lane, acc);
  }
  const DT a0 = acc[0], a1 = acc[1];
  if (lane == 0) {
    cnt.out_e += (uint64_t)(Dn ? b - a : 0);
    cnt.heavy++;
  }
  DT *part = reinterpret_cast<DT *>(p.w.partial) + (size_t)item * kK;
  part[lane] = a0;
  part[32 + lane] = a1;
  const unsigned ticket = chunk_ticket(p.w.harrive + r.h, lane);
  if (ticket != (unsigned)(nch - 1)) return;
  const DT *pp = reinterpret_cast<const DT *>(p.w.partial);
  DT t0 = 0, t1 = 0;
#pragma unroll 4
  for (int64_t cc = r.first; cc < r.first + nch; ++cc) {
    t0 += ldcg(pp + (size_t)cc * kK + lane);
    t1 += ldcg(pp + (size_t)cc * kK + 32 + lane);
  }
  const double contrib = dense_close<DT>(p, l, v, F, t0, t1, s_lo, s_hi, lane);
  red[lane] = contrib;
  __syncwarp();
  if (lane == 0) {
    double sum = 0.0;
    for (int j = 0; j < kWarp; ++j) sum += red[j];
    if (sum != 0.0) p.bc[v] = ldcg(p.bc + v) + sum;
    p.w.vis[v] = 0;
    p.w.harrive[r.h] = 0;
    cnt.entries++;
  }
  __syncwarp();
}

// Clears one level's mask array (n words) with the whole grid.
__device__ __forceinline__ void clear_level(uint64_t *m, int n, int64_t gtid, int64_t nthr) {
  for (int64_t i = gtid; i < n; i += nthr) m[i] = 0;
}

template <typename DT>
__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) dense_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DenseSmem &sm = *reinterpret_cast<DenseSmem *>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * kBlock;
  Ctl *ctl = p.w.ctl;
  const int n = p.g.n;
  uint64_t *const lm = p.w.lm;
  unsigned long long *acc = sm.acc[wib];
  double *red = &sm.red[wib][0][0];
  Counters cnt;

  if (read_err(ctl)) return;
  const int s_lo = lane < p.k ? __ldg(p.src + lane) : -1;
  const int s_hi = lane + 32 < p.k ? __ldg(p.src + lane + 32) : -1;

  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      ctl->ovf[0] = 0;
      ctl->nlevels = 0;
      p.w.hpack[0] = 0;
      p.w.hpack[1] = 0;
      p.w.hoff[0] = 0;
    }
    __syncthreads();
    if (threadIdx.x < p.k) {
      const int j = threadIdx.x;
      const int s = __ldg(p.src + j);
      atomicOr(reinterpret_cast<unsigned long long *>(p.w.vis + s), 1ull << j);
      const uint64_t old = atomicOr(reinterpret_cast<unsigned long long *>(lm + s), 1ull << j);
      const int nch = __ldg(p.g.nchunks + s);
      if (old == 0 && nch > 0) heavy_enqueue(p, 0, 0, s, nch);
    }
  }
  if (p.skip_block == (int)blockIdx.x) return; // failure-injection hook: never arrives
  if (!grid_sync(ctl, p.timeout_ns)) return;

  const int64_t n_groups = ((int64_t)n + kGroup - 1) / kGroup;

  // ---- forward sweep ---------------------------------------------------------
  int L = 0;
  int step = 0;
  HeavyLevel hl;
  hl.hoff = 0;
  for (int l = 0;; ++l) {
    const uint64_t *A = lm + (size_t)l * n;
    uint64_t *Bn = (l + 1 < p.w.dmax) ? lm + (size_t)(l + 1) * n : nullptr;
    const uint64_t *Pm = l > 0 ? lm + (size_t)(l - 1) * n : nullptr;
    const unsigned long long hp = ldcg(p.w.hpack + l);
    hl.lvl = l;
    hl.nheavy = (int64_t)(hp >> 32);
    hl.nhc = (int64_t)(hp & 0xffffffffull);
    hl.hoff_next = hl.hoff + hl.nheavy;
    if (gtid == 0) {
      p.w.hoff[l] = hl.hoff;
      p.w.hpack[l + 2] = 0;
    }
    const int64_t items = hl.nhc + n_groups;
    const int64_t my_items = items > blockIdx.x ? (items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    trace_step(p, step, l, items, hl.nhc, gtid);
    if (threadIdx.x == 0) sm.next = 0;
    __syncthreads();
    bool any_new = false;
    while (true) {
      unsigned long long k = 0;
      if (lane == 0) k = atomicAdd(&sm.next, 1ull);
      k = __shfl_sync(kFull, k, 0);
      if ((int64_t)k >= my_items) break;
      const int64_t item = (int64_t)blockIdx.x + (int64_t)k * gridDim.x;
      if (item < hl.nhc)
        fwd_chunk<DT>(p, hl, item, A, Bn, Pm, acc, lane, cnt, any_new);
      else
        fwd_group<DT>(p, hl, (item - hl.nhc) * kGroup, A, Bn, Pm, acc, sm.ovf[wib], lane, cnt,
                      any_new);
    }
    if (__ballot_sync(kFull, any_new) && lane == 0) p.w.lvl_flag[l + 1] = 1;
    if (!grid_sync(ctl, p.timeout_ns)) return;
    ++step;
    hl.hoff = hl.hoff_next;
    if (ldcg(p.w.lvl_flag + l + 1) == 0) {
      L = l + 1;
      break;
    }
  }

  if (gtid == 0) {
    ctl->nlevels = L;
    atomicMax(p.job_cnt + CNT_MAXLEV, (unsigned long long)L);
    atomicAdd(p.job_cnt + CNT_LEVELS, (unsigned long long)L);
    const uint64_t ob = ldcg(&ctl->ovf[0]);
    for (int j = 0; j < p.k; ++j)
      if ((ob >> j) & 1ull) p.ovf_flags[p.src_base + j] = 1;
  }

  // ---- backward sweep ------------------------------------------------------------
  for (int l = L - 1; l >= 0; --l) {
    const uint64_t *A = lm + (size_t)l * n;
    const uint64_t *Dn = (l + 1 < L) ? lm + (size_t)(l + 1) * n : nullptr;
    const unsigned long long hp = ldcg(p.w.hpack + l);
    HeavyLevel bl;
    bl.lvl = l;
    bl.hoff = ldcg(p.w.hoff + l);
    bl.nheavy = (int64_t)(hp >> 32);
    bl.nhc = (int64_t)(hp & 0xffffffffull);
    bl.hoff_next = 0;
    const int64_t items = bl.nhc + n_groups;
    const int64_t my_items = items > blockIdx.x ? (items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    trace_step(p, step, -1 - l, items, bl.nhc, gtid);
    if (l + 2 <= L - 1) clear_level(lm + (size_t)(l + 2) * n, n, gtid, nthr);
    if (threadIdx.x == 0) sm.next = 0;
    __syncthreads();
    while (true) {
      unsigned long long k = 0;
      if (lane == 0) k = atomicAdd(&sm.next, 1ull);
      k = __shfl_sync(kFull, k, 0);
      if ((int64_t)k >= my_items) break;
      const int64_t item = (int64_t)blockIdx.x + (int64_t)k * gridDim.x;
      if (item < bl.nhc)
        bwd_chunk<DT>(p, bl, item, A, Dn, acc, red, s_lo, s_hi, lane, cnt);
      else
        bwd_group<DT>(p, l, (item - bl.nhc) * kGroup, A, Dn, acc, red, s_lo, s_hi, lane, cnt);
    }
    if (!grid_sync(ctl, p.timeout_ns)) return;
    ++step;
  }
  trace_step(p, step, 1 << 20, 0, 0, gtid); // end marker

  // ---- leave the workspace clean for the next batch ---------------------------------
  clear_level(lm, n, gtid, nthr);
  if (L >= 2) clear_level(lm + (size_t)n, n, gtid, nthr);
  if (gtid == 0)
    for (int l = 0; l <= L; ++l) p.w.lvl_flag[l] = 0;
  // per-lane counters: reduce across the warp, one atomic per warp and counter
  unsigned long long e = cnt.entries, r = cnt.reached;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e += __shfl_down_sync(kFull, e, off);
    r += __shfl_down_sync(kFull, r, off);
  }
  if (lane == 0) {
    atomicAdd(p.job_cnt + CNT_ENTRIES, e);
    atomicAdd(p.job_cnt + CNT_OUT_EDGES, cnt.out_e);
    atomicAdd(p.job_cnt + CNT_IN_EDGES, cnt.in_e);
    atomicAdd(p.job_cnt + CNT_DAG, cnt.dag);
    atomicAdd(p.job_cnt + CNT_REACHED, r);
    atomicAdd(p.job_cnt + CNT_HEAVY, cnt.heavy);
  }
}

template <typename K> int dense_grid(K kernel, int device) {
  int per_sm = 0, sms = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(DenseSmem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, sizeof(DenseSmem)) !=
      cudaSuccess)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <typename K> cudaError_t dense_launch(K kernel, const KParams &p, int grid,
                                               cudaStream_t st) {
  void *args[] = {const_cast<KParams *>(&p)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kernel), dim3(grid),
                                     dim3(kBlock), args, sizeof(DenseSmem), st);
}

} // namespace

cudaError_t launch_dense(const KParams &p, bool fp64, int grid, cudaStream_t st) {
  return fp64 ? dense_launch(dense_kernel<double>, p, grid, st)
              : dense_launch(dense_kernel<float>, p, grid, st);
}

int max_grid_dense(bool fp64, int device) {
  return fp64 ? dense_grid(dense_kernel<double>, device) : dense_grid(dense_kernel<float>, device);
}

} // namespace bcgpu
