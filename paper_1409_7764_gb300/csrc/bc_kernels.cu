// Kernel translation unit of the GB300 betweenness-centrality library: the
// batched kernels in their standard instantiations (one workspace layout per
// mask width), the one-source plain kernels and the small helper kernels,
// with their host launchers.  The batched sweeps
// themselves are in bc_batch.cuh.
#include "bc_batch.cuh"

#include <cstdio>

namespace bcgpu {

namespace {

// ---------------------------------------------------------------------------
// plain kernel: one source, lanes over edges
// ---------------------------------------------------------------------------

__device__ __forceinline__ void warp_sat_sum(uint64_t &v, bool &o) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t w = __shfl_down_sync(kFull, v, off);
    const bool ow = __shfl_down_sync(kFull, (int)o, off) != 0;
    o = o || ow;
    sat_add(v, w, o);
  }
}


__device__ __forceinline__ void plain_discover(const KParams &p, const LevelView &lv, int64_t eb,
                                               int64_t ee, int lane) {
  for (int64_t base = eb; base < ee; base += kWarp) {
    const int64_t e = base + lane;
    bool isnew = false;
    int x = 0;
    if (e < ee) {
      x = __ldg(p.g.col_idx + e);
      if (ldcg(p.w.d + x) < 0) isnew = (atomicCAS(p.w.d + x, -1, lv.lvl + 1) == -1);
    }
    enqueue_new(p, lv, isnew, x, lane);
  }
}

__device__ __forceinline__ void plain_pull_sigma(const KParams &p, int lvl, int64_t eb,
                                                 int64_t ee, int lane, uint64_t &s, bool &o,
                                                 unsigned long long &dag) {
  unsigned long long nd = 0;
  for (int64_t e = eb + lane; e < ee; e += kWarp) {
    const int u = __ldg(p.g.in_idx + e);
    if (ldcg(p.w.d + u) == lvl - 1) {
      sat_add(s, ldcg(p.w.sigma + u), o);
      ++nd;
    }
  }
  dag += nd;
}

template <typename DT>
__device__ __forceinline__ DT plain_pull_delta(const KParams &p, int lvl, int64_t eb, int64_t ee,
                                               int lane) {
  const DT *cdep = reinterpret_cast<const DT *>(p.w.cdep);
  DT a = 0;
  for (int64_t e = eb + lane; e < ee; e += kWarp) {
    const int x = __ldg(p.g.col_idx + e);
    if (ldcg(p.w.d + x) == lvl + 1) a += ldcg(cdep + x);
  }
  return a;
}

template <typename DT>
__device__ __forceinline__ void plain_finish(const KParams &p, int lvl, int v, DT acc, int s) {
  // lane 0 only
  const uint64_t sg = ldcg(p.w.sigma + v);
  const DT sf = u64_to<DT>(sg);
  const DT dl = sf * acc;
  reinterpret_cast<DT *>(p.w.cdep)[v] = (DT(1) + dl) / sf;
  p.w.sigma[v] = 0;
  if (v != s && dl != DT(0)) p.bc[v] = ldcg(p.bc + v) + (double)dl;
  if (p.dbg_d) {
    p.dbg_d[v] = lvl;
    p.dbg_sigma[v] = sg;
    p.dbg_delta[v] = (double)dl;
  }
}

// One source through both sweeps in the given scope: the whole grid of a
// cooperative launch (grid barriers between levels), or one thread block
// (block barriers; small graphs, where many such launches run at once).
template <typename DT, typename Scope>
__device__ __forceinline__ void plain_body(const KParams &p, const Scope sc) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t)sc.rank() * kWarpsPerBlock + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)sc.size() * kWarpsPerBlock;
  const int64_t gtid = (int64_t)sc.rank() * kBlock + threadIdx.x;
  const int64_t nthr = (int64_t)sc.size() * kBlock;
  Ctl *ctl = p.w.ctl;
  Counters cnt;
  if (read_err(ctl)) return;
  const int s = __ldg(p.src);

  if (sc.rank() == 0 && threadIdx.x == 0) {
    ctl->tail = 1;
    ctl->ovf[0] = 0;
    for (int i = 0; i < 4; ++i) ctl->work[i] = 0;
    p.w.qv[0] = s;
    p.w.d[s] = 0;
    p.w.qoff[0] = 0;
    p.w.qoff[1] = 1;
    p.w.hoff[0] = 0;
    p.w.hpack[1] = 0;
    const int nch = __ldg(p.g.nchunks + s);
    p.w.hpack[0] = nch > 0 ? ((1ull << 32) | (unsigned long long)nch) : 0ull;
    if (nch > 0) {
      p.w.hq_e[0] = 0;
      p.w.hq_c[0] = 0;
    }
  }
  if (Scope::kGrid && p.skip_block == sc.rank()) return; // failure-injection hook
  if (!sc.sync(ctl, p.timeout_ns)) return;

  LevelView lv;
  lv.lvl = 0;
  lv.lo = 0;
  lv.hi = 1;
  lv.hoff = 0;
  int L = 0;
  int step = 0;
  while (true) {
    const int l = lv.lvl;
    const unsigned long long hp = ldcg(p.w.hpack + l);
    lv.nheavy = (int64_t)(hp >> 32);
    lv.nhc = (int64_t)(hp & 0xffffffffull);
    lv.hoff_next = lv.hoff + lv.nheavy;
    if (gtid == 0) {
      p.w.hoff[l] = lv.hoff;
      p.w.hpack[l + 2] = 0;
    }
    zero_ring_ahead(ctl, step, gtid);
    unsigned long long *ctr = &ctl->work[step & 3];
    const int64_t total = lv.nhc + (lv.hi - lv.lo);
    trace_step(p, step, l, total, lv.nhc, gtid);
    HeavyCursor hc;
    const int grab = p.grab;
    const int64_t stat = nwarps * grab;
    int64_t base = gwarp * grab;
    while (base < total) {
      const int64_t next = BC_PREFETCH_GROUPS ? next_items(ctr, total, stat, grab, lane) : 0;
      const int64_t end = base + grab < total ? base + grab : total;
      for (int64_t item = base; item < end; ++item) {
        if (item < lv.nhc) {
          hc.seek(p, lv, item, lane);
          const int64_t h = hc.h;
          const int64_t e = ldcg(p.w.hq_e + h);
          const int w = ldcg(p.w.qv + e);
          const int nch = __ldg(p.g.nchunks + w);
          const int64_t c = item - hc.first;
          const int64_t is = __ldg(p.g.in_ptr + w), ie = __ldg(p.g.in_ptr + w + 1);
          const int64_t rs = __ldg(p.g.row_ptr + w), re = __ldg(p.g.row_ptr + w + 1);
          const int64_t indeg = ie - is, tot = indeg + (re - rs);
          const int64_t a = c * tot / nch, b = (c + 1) * tot / nch;
          uint64_t sv = 0;
          bool o = false;
          if (l > 0 && a < indeg)
            plain_pull_sigma(p, l, is + a, is + (b < indeg ? b : indeg), lane, sv, o, cnt.dag);
          warp_sat_sum(sv, o);
          if (b > indeg)
            plain_discover(p, lv, rs + (a > indeg ? a - indeg : 0), rs + (b - indeg), lane);
          if (lane == 0) {
            cnt.in_e += (uint64_t)((b < indeg ? b : indeg) - (a < indeg ? a : indeg));
            cnt.out_e += (uint64_t)((b > indeg ? b - indeg : 0) - (a > indeg ? a - indeg : 0));
            cnt.heavy++;
            reinterpret_cast<uint64_t *>(p.w.partial)[item] = sv;
            p.w.partial_ovf[item] = o ? 1ull : 0ull;
          }
          const unsigned ticket = chunk_ticket(p.w.harrive + h, lane);
          if (ticket == (unsigned)(nch - 1) && lane == 0) {
            const int64_t c0 = hc.first;
            uint64_t t = 0;
            bool q = false;
            if (l == 0) {
              t = 1;
            } else {
              const uint64_t *pp = reinterpret_cast<const uint64_t *>(p.w.partial);
#pragma unroll 4
              for (int64_t cc = c0; cc < c0 + nch; ++cc) {
                sat_add(t, ldcg(pp + cc), q);
                q = q || ldcg(p.w.partial_ovf + cc) != 0;
              }
            }
            p.w.sigma[w] = t;
            if (q) atomicOr(&ctl->ovf[0], 1ull);
            p.w.harrive[h] = 0;
            cnt.entries++;
            cnt.reached++;
          }
        } else {
          const int64_t e = lv.lo + (item - lv.nhc);
          const int w = ldcg(p.w.qv + e);
          if (__ldg(p.g.nchunks + w) > 0) continue;
          const int64_t is = __ldg(p.g.in_ptr + w), ie = __ldg(p.g.in_ptr + w + 1);
          const int64_t rs = __ldg(p.g.row_ptr + w), re = __ldg(p.g.row_ptr + w + 1);
          uint64_t sv = 0;
          bool o = false;
          if (l > 0) plain_pull_sigma(p, l, is, ie, lane, sv, o, cnt.dag);
          warp_sat_sum(sv, o);
          if (lane == 0) {
            p.w.sigma[w] = (l == 0) ? 1ull : sv;
            if (o) atomicOr(&ctl->ovf[0], 1ull);
            cnt.entries++;
            cnt.reached++;
            cnt.in_e += (uint64_t)(l > 0 ? ie - is : 0);
            cnt.out_e += (uint64_t)(re - rs);
          }
          plain_discover(p, lv, rs, re, lane);
        }
      }
      base = BC_PREFETCH_GROUPS ? next : next_items(ctr, total, stat, grab, lane);
    }
    if (!sc.sync(ctl, p.timeout_ns, p.w.qoff + l + 2)) return;
    ++step;
    const int64_t nh = ldcg(p.w.qoff + l + 2);
    if (nh == lv.hi) {
      L = l + 1;
      break;
    }
    lv.lo = lv.hi;
    lv.hi = nh;
    lv.hoff = lv.hoff_next;
    lv.lvl = l + 1;
  }
  if (gtid == 0) {
    ctl->nlevels = L;
    atomicMax(p.job_cnt + CNT_MAXLEV, (unsigned long long)L);
    atomicAdd(p.job_cnt + CNT_LEVELS, (unsigned long long)L);
    if (ldcg(&ctl->ovf[0])) p.ovf_flags[p.src_base] = 1;
  }

  for (int l = L - 1; l >= 0; --l) {
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
      for (int64_t i = zlo + gtid; i < zhi; i += nthr) p.w.d[ldcg(p.w.qv + i)] = -1;
    }
    const bool deepest = (l == L - 1);
    unsigned long long *ctr = &ctl->work[step & 3];
    const int64_t total = bl.nhc + (bl.hi - bl.lo);
    trace_step(p, step, -1 - l, total, bl.nhc, gtid);
    HeavyCursor hc;
    const int grab = p.grab;
    const int64_t stat = nwarps * grab;
    int64_t base = gwarp * grab;
    while (base < total) {
      const int64_t next = BC_PREFETCH_GROUPS ? next_items(ctr, total, stat, grab, lane) : 0;
      const int64_t end = base + grab < total ? base + grab : total;
      for (int64_t item = base; item < end; ++item) {
        if (item < bl.nhc) {
          hc.seek(p, bl, item, lane);
          const int64_t h = hc.h;
          const int64_t e = ldcg(p.w.hq_e + h);
          const int v = ldcg(p.w.qv + e);
          const int nch = __ldg(p.g.nchunks + v);
          const int64_t c = item - hc.first;
          const int64_t rs = __ldg(p.g.row_ptr + v), re = __ldg(p.g.row_ptr + v + 1);
          const int64_t od = re - rs;
          const int64_t a = c * od / nch, b = (c + 1) * od / nch;
          DT acc = 0;
          if (!deepest) acc = plain_pull_delta<DT>(p, l, rs + a, rs + b, lane);
          acc = warp_sum<DT>(acc);
          if (lane == 0) {
            cnt.out_e += (uint64_t)(deepest ? 0 : b - a);
            cnt.heavy++;
            reinterpret_cast<DT *>(p.w.partial)[item] = acc;
          }
          const unsigned ticket = chunk_ticket(p.w.harrive + h, lane);
          if (ticket == (unsigned)(nch - 1) && lane == 0) {
            const int64_t c0 = hc.first;
            const DT *pp = reinterpret_cast<const DT *>(p.w.partial);
            DT t = 0;
#pragma unroll 4
            for (int64_t cc = c0; cc < c0 + nch; ++cc) t += ldcg(pp + cc);
            plain_finish<DT>(p, l, v, t, s);
            p.w.harrive[h] = 0;
          }
        } else {
          const int64_t e = bl.lo + (item - bl.nhc);
          const int v = ldcg(p.w.qv + e);
          if (__ldg(p.g.nchunks + v) > 0) continue;
          DT acc = 0;
          if (!deepest) {
            const int64_t rs = __ldg(p.g.row_ptr + v), re = __ldg(p.g.row_ptr + v + 1);
            acc = plain_pull_delta<DT>(p, l, rs, re, lane);
            if (lane == 0) cnt.out_e += (uint64_t)(re - rs);
          }
          acc = warp_sum<DT>(acc);
          if (lane == 0) plain_finish<DT>(p, l, v, acc, s);
        }
      }
      base = BC_PREFETCH_GROUPS ? next : next_items(ctr, total, stat, grab, lane);
    }
    if (!sc.sync(ctl, p.timeout_ns)) return;
    ++step;
  }
  trace_step(p, step, 1 << 20, 0, 0, gtid); // end marker
  {
    const int64_t q2 = L >= 2 ? ldcg(p.w.qoff + 2) : ldcg(p.w.qoff + 1);
    for (int64_t i = gtid; i < q2; i += nthr) p.w.d[ldcg(p.w.qv + i)] = -1;
  }
  flush_counters(p.job_cnt, cnt, lane);
}

template <typename DT>
__global__ void __launch_bounds__(kBlock) plain_kernel(const KParams p) {
  plain_body<DT>(p, GridScope());
}

// One source in one thread block: the small-graph form of the one-source
// launch; the host issues such launches on several streams at once, each
// stream adding into its own BC partial vector.  The launch carries only the
// stream slot's parameters (in device memory) and the source's position b
// in the job, which keeps the host's cost per launch low: on small graphs
// the rate of launches bounds this schedule.
template <typename DT>
__global__ void __launch_bounds__(kBlock) plain_block_kernel(const KParams *__restrict__ slots,
                                                             int slot, int64_t b) {
  __shared__ KParams sp;
  constexpr int kWords = (int)(sizeof(KParams) / sizeof(unsigned long long));
  static_assert(sizeof(KParams) % sizeof(unsigned long long) == 0, "copied in 8-byte words");
  const unsigned long long *from = reinterpret_cast<const unsigned long long *>(slots + slot);
  unsigned long long *to = reinterpret_cast<unsigned long long *>(&sp);
  for (int i = threadIdx.x; i < kWords; i += blockDim.x) to[i] = from[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    sp.src += b;
    sp.src_base = b;
    if (sp.dbg_d) {
      sp.dbg_d += b * sp.g.n;
      sp.dbg_sigma += b * sp.g.n;
      sp.dbg_delta += b * sp.g.n;
    }
  }
  __syncthreads();
  plain_body<DT>(sp, CtaScope());
}

// out[v] (+)= sum over parts of parts[part][v], parts in order (deterministic).
__global__ void sum_parts_kernel(const double *__restrict__ parts, int nparts, int64_t n,
                                 double *__restrict__ out, bool add) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    double t = add ? out[v] : 0.0;
    for (int i = 0; i < nparts; ++i) t += parts[(size_t)i * n + v];
    out[v] = t;
  }
}

// The first device error of any of the control blocks, into the first one.
__global__ void gather_err_kernel(Ctl *first, size_t stride_bytes, int count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (first->err) return;
  for (int i = 1; i < count; ++i) {
    const Ctl *c = reinterpret_cast<const Ctl *>(reinterpret_cast<const char *>(first) +
                                                 stride_bytes * (size_t)i);
    if (c->err) {
      first->err = c->err;
      return;
    }
  }
}

__global__ void scale_kernel(const double *__restrict__ in, double *__restrict__ out, int64_t n,
                             double factor) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * factor;
}

// Sampled-source estimate from the sums of the per-source terms and of their
// squares over k sources: est = f*n*m, err = f*n*sqrt((1 - k/n) S2 / k) with
// m the mean, S2 = (sum of squares - k m^2)/(k - 1) the sample variance
// (clamped at 0 against rounding) and f the output scale; err is NaN for
// k < 2, and the finite-population factor is clamped at 0 for k > n.
__global__ void estimate_kernel(const double *__restrict__ sum, const double *__restrict__ sumsq,
                                int64_t n, int64_t k, double factor, double *__restrict__ est,
                                double *__restrict__ err) {
  const double nn = (double)n, kk = (double)k;
  const double fpc = k >= n ? 0.0 : 1.0 - kk / nn;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double m = k > 0 ? sum[v] / kk : 0.0;
    est[v] = factor * nn * m;
    if (k < 2) {
      err[v] = nan("");
    } else {
      double s2 = (sumsq[v] - kk * m * m) / (kk - 1.0);
      if (s2 < 0.0) s2 = 0.0;
      err[v] = factor * nn * sqrt(fpc * s2 / kk);
    }
  }
}

// Largest err[v]/est[v] over vertices with est[v] >= min_est (> 0), as the
// bit pattern of a non-negative double (which orders like the value).
__global__ void max_rel_err_kernel(const double *__restrict__ est, const double *__restrict__ err,
                                   int64_t n, double min_est, unsigned long long *out) {
  double r = 0.0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double e = est[v];
    if (e >= min_est && e > 0.0) {
      const double q = err[v] / e;
      r = q > r ? q : r;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_down_sync(kFull, r, off);
    r = o > r ? o : r;
  }
  if ((threadIdx.x & 31) == 0 && r > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(r));
}

// Adds a finished job's per-vertex sums into running accumulators, unless
// the job recorded a device error (then its sums may be partial).
__global__ void accumulate_kernel(double *__restrict__ acc, double *__restrict__ acc2,
                                  const double *__restrict__ add, const double *__restrict__ add2,
                                  int64_t n, const int *err) {
  if (*reinterpret_cast<const volatile int *>(err) != 0) return;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    acc[v] += add[v];
    acc2[v] += add2[v];
  }
}

template <typename K> int max_grid_for(K kernel, int device) {
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <typename K> cudaError_t coop_launch(K kernel, const KParams &p, int grid,
                                              cudaStream_t st) {
  void *args[] = {const_cast<KParams *>(&p)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kernel), dim3(grid),
                                     dim3(kBlock), args, 0, st);
}

template <bool SQ, typename CT>
cudaError_t launch_batch_sq(const KParams &p, bool fp64, int grid, cudaStream_t st, int words) {
  switch (words) {
    case 1:
      return fp64 ? coop_launch(batch_kernel<double, 1, SQ, CT>, p, grid, st)
                  : coop_launch(batch_kernel<float, 1, SQ, CT>, p, grid, st);
    case 2:
      return fp64 ? coop_launch(batch_kernel<double, 2, SQ, CT>, p, grid, st)
                  : coop_launch(batch_kernel<float, 2, SQ, CT>, p, grid, st);
    case 4:
      return fp64 ? coop_launch(batch_kernel<double, 4, SQ, CT>, p, grid, st)
                  : coop_launch(batch_kernel<float, 4, SQ, CT>, p, grid, st);
    default:
      return cudaErrorInvalidValue;
  }
}

} // namespace

// The squared-term accumulation of the estimator is a separate
// instantiation, so plain BC jobs carry none of its code.
// Estimator jobs keep 64-bit counts.
cudaError_t launch_batch(const KParams &p, bool fp64, int grid, cudaStream_t st, int words,
                         bool counts32) {
  if (p.bc2) return launch_batch_sq<true, uint64_t>(p, fp64, grid, st, words);
  return counts32 ? launch_batch_sq<false, uint32_t>(p, fp64, grid, st, words)
                  : launch_batch_sq<false, uint64_t>(p, fp64, grid, st, words);
}

cudaError_t launch_plain(const KParams &p, bool fp64, int grid, cudaStream_t st) {
  return fp64 ? coop_launch(plain_kernel<double>, p, grid, st)
              : coop_launch(plain_kernel<float>, p, grid, st);
}

cudaError_t launch_plain_block(const KParams *slots, int slot, int64_t b, bool fp64,
                               cudaStream_t st) {
  if (fp64) plain_block_kernel<double><<<1, kBlock, 0, st>>>(slots, slot, b);
  else plain_block_kernel<float><<<1, kBlock, 0, st>>>(slots, slot, b);
  return cudaGetLastError();
}

cudaError_t launch_sum_parts(const double *parts, int nparts, int64_t n, double *out,
                             cudaStream_t st, bool add_to_out) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  sum_parts_kernel<<<grid, 256, 0, st>>>(parts, nparts, n, out, add_to_out);
  return cudaGetLastError();
}

template <typename K>
cudaError_t coop_launch_multi(K kernel, const MultiParams &mp, cudaStream_t st) {
  void *args[] = {const_cast<MultiParams *>(&mp)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kernel),
                                     dim3(mp.groups * mp.gsize), dim3(kBlock), args, 0, st);
}

template <typename CT>
cudaError_t launch_multi_ct(const MultiParams &mp, bool fp64, int words, cudaStream_t st) {
  switch (words) {
    case 1:
      return fp64 ? coop_launch_multi(multi_batch_kernel<double, 1, false, CT>, mp, st)
                  : coop_launch_multi(multi_batch_kernel<float, 1, false, CT>, mp, st);
    case 2:
      return fp64 ? coop_launch_multi(multi_batch_kernel<double, 2, false, CT>, mp, st)
                  : coop_launch_multi(multi_batch_kernel<float, 2, false, CT>, mp, st);
    case 4:
      return fp64 ? coop_launch_multi(multi_batch_kernel<double, 4, false, CT>, mp, st)
                  : coop_launch_multi(multi_batch_kernel<float, 4, false, CT>, mp, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_multi(const MultiParams &mp, bool fp64, int words, bool counts32,
                         cudaStream_t st) {
  return counts32 ? launch_multi_ct<uint32_t>(mp, fp64, words, st)
                  : launch_multi_ct<uint64_t>(mp, fp64, words, st);
}

cudaError_t launch_gather_err(Ctl *first, size_t stride_bytes, int count, cudaStream_t st) {
  gather_err_kernel<<<1, 32, 0, st>>>(first, stride_bytes, count);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double *in, double *out, int64_t n, double factor,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  scale_kernel<<<grid, 256, 0, st>>>(in, out, n, factor);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(double *acc, double *acc2, const double *add, const double *add2,
                              int64_t n, const int *err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  accumulate_kernel<<<grid, 256, 0, st>>>(acc, acc2, add, add2, n, err);
  return cudaGetLastError();
}

cudaError_t launch_estimate(const double *sum, const double *sumsq, int64_t n, int64_t k,
                            double factor, double *est, double *err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  estimate_kernel<<<grid, 256, 0, st>>>(sum, sumsq, n, k, factor, est, err);
  return cudaGetLastError();
}

cudaError_t launch_max_rel_err(const double *est, const double *err, int64_t n, double min_est,
                               unsigned long long *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 1024) grid = 1024;
  max_rel_err_kernel<<<grid, 256, 0, st>>>(est, err, n, min_est, out);
  return cudaGetLastError();
}

int max_grid_batch(bool fp64, int device, int words) {
  switch (words) {
    case 1:
      return fp64 ? max_grid_for(batch_kernel<double, 1, false, uint64_t>, device)
                  : max_grid_for(batch_kernel<float, 1, false, uint64_t>, device);
    case 2:
      return fp64 ? max_grid_for(batch_kernel<double, 2, false, uint64_t>, device)
                  : max_grid_for(batch_kernel<float, 2, false, uint64_t>, device);
    case 4:
      return fp64 ? max_grid_for(batch_kernel<double, 4, false, uint64_t>, device)
                  : max_grid_for(batch_kernel<float, 4, false, uint64_t>, device);
    default:
      return 0;
  }
}

int max_grid_plain(bool fp64, int device) {
  return fp64 ? max_grid_for(plain_kernel<double>, device)
              : max_grid_for(plain_kernel<float>, device);
}

} // namespace bcgpu
