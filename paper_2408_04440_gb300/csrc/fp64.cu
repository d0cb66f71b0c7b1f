// fp64.cu -- FP64 kernels of the tile Cholesky ("Advancements in Dense Linear
// Algebra": POTRF on the diagonal tile, TRSM on the panel, SYRK/GEMM on the
// trailing tiles), the TRMM that draws emulations ("Generating Emulations",
// xi = V z) and the tile-blocked triangular solves.
//
// GB300 runs FP64 on the SIMT pipe at about 2 DFMA per clock per SM (the FP64
// MMA path measured slower), so these kernels are FP64-issue bound: the
// register/shared-memory blocking below only has to keep that pipe busy.
#include <climits>
#include <vector>

#include "emu_internal.h"
#include "tc.cuh"

namespace {

constexpr int B = 32;  // inner block of the diagonal-tile POTRF and the TRSM

__device__ inline bool failed(const int *st) {
  return *((volatile const int *)st) != DEV_OK;
}

// ------------------------------------------------------------ POTRF (tile)
// FP64 Cholesky of one diagonal tile D (nb x nb, column-major) as a
// persistent dataflow kernel over 16 x 16 blocks.  Tasks:
//   LT(s)      solve the sub-diagonal block X_{s,s-1} = D_{s,s-1} L_{s-1,s-1}^{-T}
//              (after applying panel s-2 to it), apply it to the diagonal
//              block (s,s), and factor that block (the leaf);
//   TRSM(r,s)  r >= s+2: apply panel s-1 to block (r,s), then solve it;
//   UPD(r,c,s) c >= s+2: D_rc -= X_rs X_cs^T.
// A block's last update is fused into the task that finalises it, so the
// critical chain is LT(s) -> LT(s+1): one task per 16-column step.  Tasks
// are listed in a topological, lookahead-first order and fetched by the CTAs
// through an atomic counter.  state[r*nbb + c] counts completed operations on
// block (r,c) (final value c+1).  Because tasks are fetched in topological
// order the earliest unfinished task always has its inputs ready, so the
// kernel makes progress whatever number of CTAs is resident.  Every wait is
// bounded (status DEV_TIMEOUT) and every CTA leaves as soon as the status
// word reports a failure.  Data written by other CTAs is read through L2.
// On GB300 an FP64 warp instruction holds its SM sub-partition's FP64 pipe
// for 64 cycles however many lanes are active, and an FP64 rsqrt costs ~430.
// So the leaf spreads the block over four warps (one per sub-partition),
// eliminates without square roots (pivot reciprocals on the chain, scaling
// by rsqrt once at the end), and the solves use L scaled by the pivot
// reciprocals (one dependent FMA per substitution step).  LT(s) publishes
// X_{s,s-1} before its leaf, so that LT(s+1) applies panel s-1 to block
// (s+1, s) while the leaf runs.
constexpr int PB = 16;
enum { T_LT = 0, T_TRSM = 1, T_UPD = 2, T_MASTER = 3, T_HELP = 5, T_HELP2 = 6 };
// wait bound in SM clock cycles (about 2 s at 2 GHz)
constexpr long long kDagWaitCycles = 4000000000ll;

// GPU-scope acquire-release fence.  A block publishes data with its threads'
// stores, a barrier, then one thread's fence and flag write (the fence is
// cumulative over the stores the barrier ordered before it); a reader's
// thread polls the flag, fences, and a barrier passes the acquisition on.
__device__ inline void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ inline uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Test hooks of the timeout path (emu_test_wait_hook): the bound of the flag
// waits, and one flag index that every wait treats as never set.
__constant__ long long c_dag_wait_cycles = kDagWaitCycles;
__constant__ int c_dag_withhold = -1;

// Thread 0 waits until state[idx] >= v (or failure / timeout).
__device__ inline bool dag_wait(const int *state, int idx, int v, int *st) {
  volatile const int *p = state + idx;
  const bool held = idx == c_dag_withhold;
  if (!held && *p >= v) return true;
  const long long t0 = clock64(), limit = c_dag_wait_cycles;
  while (true) {
    if (!held && *p >= v) return true;
    if (*((volatile const int *)st) != DEV_OK) return false;
    if (clock64() - t0 > limit) {
      if (atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 2;
      return false;
    }
    __nanosleep(32);
  }
}

// Thread 0 waits until state[i] >= v for up to three flags (an index < 0 is
// no flag), or failure / timeout, polling every flag in each round so that
// one L2 round trip serves them all.
__device__ inline bool dag_wait3(const int *state, int i0, int v0, int i1, int v1, int i2, int v2, int *st) {
  const int w = c_dag_withhold;
  long long t0 = 0;
  for (int it = 0;; it++) {
    const int a = i0 >= 0 ? *((volatile const int *)(state + i0)) : INT_MAX;
    const int b = i1 >= 0 ? *((volatile const int *)(state + i1)) : INT_MAX;
    const int c = i2 >= 0 ? *((volatile const int *)(state + i2)) : INT_MAX;
    const bool held = (i0 >= 0 && i0 == w) || (i1 >= 0 && i1 == w) || (i2 >= 0 && i2 == w);
    if (a >= v0 && b >= v1 && c >= v2 && !held) return true;
    if (*((volatile const int *)st) != DEV_OK) return false;
    if (it == 0) {
      t0 = clock64();
    } else if (clock64() - t0 > c_dag_wait_cycles) {
      if (atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 2;
      return false;
    }
    __nanosleep(32);
  }
}
// Thread 0 of an idle CTA: waits until *flag >= v, the factor has failed,
// or the flag waits' bound has passed, whichever comes first; it sets no
// status (the waits that need the flag report a timeout themselves).
__device__ inline void idle_until(const int *flag, int v, const int *st) {
  const long long t0 = clock64();
  while (*((volatile const int *)flag) < v && *((volatile const int *)st) == DEV_OK &&
         clock64() - t0 <= c_dag_wait_cycles)
    __nanosleep(256);
}
__device__ inline bool dag_wait2(const int *state, int i0, int v0, int i1, int v1, int *st) {
  return dag_wait3(state, i0, v0, i1, v1, -1, 0, st);
}

// The leaf releases its columns in groups 0-3, 4-7, 8-11, 12-13, 14, 15
// (one barrier each, that of the group's last column): whether column j
// opens its group, and the barrier of j's group.
__host__ __device__ constexpr bool col_group_first(int j) { return j < 12 ? (j & 3) == 0 : j != 13; }
__host__ __device__ constexpr int col_group_bar(int j) { return j < 12 ? (j | 3) : (j == 12 ? 13 : j); }

// Pivot reciprocal: the hardware approximation y (relative error about
// 2^-20, measured) refined by one third-order Newton-Raphson step for 1/d,
// r = y (1 + e + e^2) with e = 1 - d y, whose truncation error e^3 is below
// 2^-59; three dependent FMAs instead of the ~7 of an FP64 rsqrt.  The
// approximation flushes subnormal inputs and results, so it is used for
// pivots in [2^-1000, 2^1000) only (pivot_in_range).
__device__ inline double pivot_rcp(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
// d positive, finite and in [2^-1000, 2^1000): biased exponent in [23, 2023).
// An integer test on the high word: FP64 comparisons occupy the FP64 pipe
// like an FMA.
__device__ inline bool pivot_in_range(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  return hi - (23u << 20) < (2000u << 20);
}

__device__ inline void bar_sync_128(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
__device__ inline void bar_sync_256(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }
__device__ inline void bar_arrive_256(int id) { asm volatile("bar.arrive %0, 256;" ::"r"(id) : "memory"); }

// ---- thread-block cluster (the single-tile chain on three SMs)
__device__ inline uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ inline uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ inline uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared object in CTA `rank`
__device__ inline uint32_t peer_addr(const void *local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_u32(local)), "r"(rank));
  return r;
}
__device__ inline void st_peer_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ inline void st_peer_s32(uint32_t addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// arrive on an mbarrier of the peer CTA; releases this thread's earlier
// stores (local and remote) at cluster scope
__device__ inline void arrive_peer(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Waits for the phase of the given parity of an mbarrier of this CTA; false
// after the wait bound or when *abort is set.  SCOPE_CLUSTER: the arrivals
// come from another CTA of the cluster (their remote stores become visible),
// polled with try_wait; else from this CTA, polled with test_wait, which
// never parks the thread (the column hand-overs inside a helper come every
// few hundred cycles).
template <bool SCOPE_CLUSTER>
__device__ inline bool wait_phase(uint64_t *bar, uint32_t parity, volatile int *abort) {
  const uint32_t a = tc::smem_u32(bar);
  long long t0 = 0;
  for (int it = 0;; it++) {
    uint32_t ok;
    if (SCOPE_CLUSTER)
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    if (ok) return true;
    if (*abort) return false;
    if (it == 0) t0 = clock64();
    else if (clock64() - t0 > c_dag_wait_cycles) return false;
  }
}
__device__ inline bool wait_from_peer(uint64_t *bar, uint32_t parity, volatile int *abort) {
  return wait_phase<true>(bar, parity, abort);
}
__device__ inline bool wait_local(uint64_t *bar, uint32_t parity, volatile int *abort) {
  return wait_phase<false>(bar, parity, abort);
}
// every thread of both CTAs; orders each CTA's remote stores before the
// other's exit
__device__ inline void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16x16 products of panel rows: sum_p A[ty][p] B[tx][p], two chains.
__device__ inline double panel_dot(const double (*A)[PB + 1], const double (*Bm)[PB + 1], int ty, int tx) {
  double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
  for (int p = 0; p < PB; p += 2) {
    acc0 += A[ty][p] * Bm[tx][p];
    acc1 += A[ty][p + 1] * Bm[tx][p + 1];
  }
  return acc0 + acc1;
}

// The leaf on warps 0..3 (u = thread index 0..127): factors the 16x16 block
// whose lower entries (i, k0) and (i, k1) the thread holds in v0, v1
// (k0 = w + 4h for warp w, half-warp h; k1 = k0 + 8).  Step j: the owner of
// column j writes the unscaled column c_j to mcol[j][*]; then every thread
// updates its trailing entries, x_ik -= c_j[i] c_j[k] / c_jj.  At the end
// L_ik = c_k[i] / sqrt(c_kk) goes to out[i][k] and 1/L_kk to rinv[k].
// Returns 0, or the 1-based column of the first non-positive pivot (the
// same in every thread; out is then not written; out may be null).  With ms
// given (the cluster form of the chain): at step j the 16 threads of rows i = u < 16 store the
// scaled column c_j[i] / c_jj (= L_ij / L_jj) into ms[j][i] and thread j the
// pivot reciprocal 1/c_jj into ms[j][16]; after columns 3, 7, 11, 13, 14 and
// 15 each arrives on the local mbarrier mb[j] (16 arrivals); at the end they
// arrive on mb[16] once rinv is written.  Every phase completes whether or not a pivot
// fails.
__device__ __forceinline__ int leaf16(int u, double v0, double v1, double (*mcol)[PB + 1], double (*out)[PB + 1],
                                      double *rinv, double (*ms)[PB + 1] = nullptr, uint64_t *mb = nullptr) {
  const int w = u >> 5, i = u & (PB - 1);
  const int k0 = w + 4 * ((u >> 4) & 1), k1 = k0 + 8;
  int fail = 0;
#pragma unroll
  for (int j = 0; j < PB; j++) {
    // the owner of the pivot computes its reciprocal once, into the padding
    // column of mcol: FP64 instructions, not lanes, are what the master's
    // SM runs short of
    if (j < 8) {
      if (k0 == j) {
        mcol[j][i] = v0;
        if (i == j && pivot_in_range(v0)) mcol[j][PB] = pivot_rcp(v0);
      }
    } else {
      if (k1 == j) {
        mcol[j][i] = v1;
        if (i == j && pivot_in_range(v1)) mcol[j][PB] = pivot_rcp(v1);
      }
    }
    bar_sync_128(1);
    // the pivot is the same in every thread: the branches are uniform
    double dj = mcol[j][j], r;
    if (pivot_in_range(dj)) {
      r = mcol[j][PB];
    } else {
      if (!(dj > 0.0)) {  // also catches NaN
        if (!fail) fail = j + 1;
        dj = 1.0;  // keep going; the result is discarded
      }
      r = 1.0 / dj;
    }
    const double tt = mcol[j][i] * r;
    // warp-uniform guards: no lane of the warp has a column > j left
    if (j < w + 4 && k0 > j && i >= k0) v0 = fma(-tt, mcol[j][k0], v0);
    if (j < w + 12 && k1 > j && i >= k1) v1 = fma(-tt, mcol[j][k1], v1);
    if (ms && u < PB) {
      ms[j][i] = tt;
      if (i == j) ms[j][PB] = r;  // the pivot reciprocal 1/c_jj
      // after columns 3, 7, 11, 13, 14, 15: one release (CTA scope) covers
      // this thread's stores since the previous one
      if ((j & 3) == 3 || j >= 13) tc::mbar_arrive(&mb[j]);
    }
  }
  if (u < PB) {
    rinv[u] = rsqrt(mcol[u][u]);
    if (ms) tc::mbar_arrive(&mb[16]);
  }
  bar_sync_128(1);
  if (!fail && out) {
    out[i][k0] = v0 * rinv[k0];  // the diagonal: c_kk / sqrt(c_kk)
    out[i][k1] = v1 * rinv[k1];
  }
  return fail;
}

// The whole chain LT(0), LT(1), ... of one tile in one CTA (task T_MASTER
// of the single-tile list), so that no step waits for another CTA's flag or
// reloads L_{s-1,s-1} from L2.  Warps 0..3 compute: the solve of block
// (s, s-1), the diagonal block minus X X^T and the leaf.  Warps 4..7 do the
// memory traffic meanwhile: they publish L_{s-1,s-1} and X_{s,s-1}, wait for
// the next step's inputs (X_{s+1,s-1} from TRSM(s+1, s-1), the updates of
// blocks (s+1, s) and (s+1, s+1) by earlier panels), load them, and apply
// panel s-1 to block (s+1, s) while the leaf runs.  Shared buffers at the
// start of step s: a = L_{s-1,s-1}, m = L_{s-1,s-1} scaled by the pivot
// reciprocals rinv, xr = block (s, s-1) after panels < s-1, xc = block (s, s)
// after panels < s-1.  Other CTAs run the TRSM / UPD tasks, which finish
// without waiting for anything but this chain and earlier tasks, so the
// chain advances as soon as one other CTA of the launch is resident.
// flags[0]: a wait failed (status already set); flags[1]: first
// non-positive pivot column in the block (1-based).
__device__ __forceinline__ void potrf_master(double *__restrict__ D, int nb, int gcol0, int *__restrict__ state,
                                             double *__restrict__ rinv_g, int *st,
                                             unsigned long long *__restrict__ trace, double (*a)[PB + 1],
                                             double (*m)[PB + 1], double (*xr)[PB + 1], double (*xc)[PB + 1],
                                             double *rinv, volatile int *flags) {
  const int nbb = nb / PB;
  const size_t ld = nb;
  const int tid = threadIdx.x, u = tid & 127;
  const bool io = tid >= 128;
  // warps 4..7: entries (ir, ic) and (ir, ic + 8), lanes along a column
  const int ir = u & (PB - 1), ic = u >> 4;
  // warps 0..3, solve: rows cr and cr + 8 of column ct (a row's 16 lanes shuffle)
  const int cr = u >> 4, ct = u & (PB - 1);
  auto gp = [&](int br, int bc, int r, int c) { return D + (size_t)(br * PB + r) + (size_t)(bc * PB + c) * ld; };
  if (tid == 0) flags[0] = flags[1] = 0;
  if (io) {
    xc[ir][ic] = __ldcg(gp(0, 0, ir, ic));
    xc[ir][ic + 8] = __ldcg(gp(0, 0, ir, ic + 8));
  }
  __syncthreads();
  for (int s = 0; s < nbb; s++) {
    const int q = s - 1, n1 = s + 1;
    unsigned long long t0 = 0, t1 = 0;
    long long c0 = 0, cx = 0, c1 = 0, cl = 0;  // trace only: SM cycles of the sub-phases
    if (trace && tid == 0) {
      t0 = gtimer();
      c0 = clock64();
    }
    if (!io) {
      // X_{s,q} = block (s, q) L_{q,q}^{-T}
      if (q >= 0) {
        double va = xr[cr][ct], vb = xr[cr + 8][ct];
#pragma unroll
        for (int j = 0; j < PB; j++) {
          const double aj = __shfl_sync(0xffffffffu, va, j, PB), bj = __shfl_sync(0xffffffffu, vb, j, PB);
          if (ct > j) {
            const double mj = m[ct][j];
            va = fma(-aj, mj, va);
            vb = fma(-bj, mj, vb);
          }
        }
        xr[cr][ct] = va * rinv[ct];
        xr[cr + 8][ct] = vb * rinv[ct];
      }
      if (trace && tid == 0) cx = clock64();
      // X_{s,q} written (the I/O warps publish it); then wait until the I/O
      // warps hold L_{q,q}, which this step's leaf overwrites: the leaf does
      // not wait for the publishing fence
      bar_arrive_256(5);
      bar_sync_256(4);
    } else {
      // publish L_{q,q} and its pivot reciprocals, read out of shared memory
      // before the compute warps' leaf overwrites them
      double la = 0.0, lb = 0.0, lr = 0.0;
      if (q >= 0) {
        la = a[ir][ic];
        lb = a[ir][ic + 8];
        if (u < PB) lr = rinv[u];
      }
      bar_arrive_256(4);
      if (q >= 0) {
        if (ir >= ic) __stcg(gp(q, q, ir, ic), la);
        if (ir >= ic + 8) __stcg(gp(q, q, ir, ic + 8), lb);
        if (u < PB) __stcg(rinv_g + q * PB + u, lr);
        bar_sync_128(2);
        if (u == 0) {
          fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
          atomicExch(&state[q * nbb + q], q + 1);
        }
      }
      bar_sync_256(5);  // X_{s,q} is in xr
    }
    if (trace && tid == 0) {
      t1 = gtimer();
      c1 = clock64();
    }
    if (!io) {
      const int i = u & (PB - 1), k0 = (u >> 5) + 4 * ((u >> 4) & 1), k1 = k0 + 8;
      double v0 = xc[i][k0], v1 = xc[i][k1];
      if (q >= 0) {
        v0 -= panel_dot(xr, xr, i, k0);
        v1 -= panel_dot(xr, xr, i, k1);
      }
      bar_arrive_256(3);  // this step's reads of xr and xc are done
      const int fail = leaf16(u, v0, v1, m, a, rinv);
      if (fail) {
        if (u == 0) flags[1] = fail;
      } else {
        bar_sync_128(1);  // a complete
        m[cr][ct] = a[cr][ct] * rinv[ct];
        m[cr + 8][ct] = a[cr + 8][ct] * rinv[ct];
      }
      if (trace && tid == 0) cl = clock64();
    } else {
      if (q >= 0) {
        // publish X_{s,q}
        __stcg(gp(s, q, ir, ic), xr[ir][ic]);
        __stcg(gp(s, q, ir, ic + 8), xr[ir][ic + 8]);
        bar_sync_128(2);
        if (u == 0) {
          fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
          atomicExch(&state[s * nbb + q], s);
        }
      }
      double pa = 0.0, pb = 0.0, ga = 0.0, gb = 0.0;
      if (n1 < nbb) {
        // block (n1, s) after panels < s-1 (and X_{n1,s-1})
        if (u == 0) {
          const bool ok = (s < 1 || dag_wait(state, n1 * nbb + (s - 1), s, st)) &&
                          dag_wait(state, n1 * nbb + s, s - 1, st);
          fence_acq_rel_gpu();
          if (!ok) flags[0] = 1;
        }
        bar_sync_128(2);
        if (!flags[0]) {
          pa = __ldcg(gp(n1, s, ir, ic));
          pb = __ldcg(gp(n1, s, ir, ic + 8));
        }
      }
      bar_sync_256(3);  // the compute warps no longer read xr / xc
      if (n1 < nbb && s >= 1 && !flags[0]) {
        xc[ir][ic] = __ldcg(gp(n1, s - 1, ir, ic));
        xc[ir][ic + 8] = __ldcg(gp(n1, s - 1, ir, ic + 8));
      }
      bar_sync_128(2);
      if (n1 < nbb && s >= 1 && !flags[0]) {
        // panel s-1 applied to block (n1, s): X_{n1,s-1} X_{s,s-1}^T
        pa -= panel_dot(xc, xr, ir, ic);
        pb -= panel_dot(xc, xr, ir, ic + 8);
      }
      if (n1 < nbb) {
        // block (n1, n1) after panels < s
        if (u == 0) {
          const bool ok = !flags[0] && dag_wait(state, n1 * nbb + n1, s, st);
          fence_acq_rel_gpu();
          if (!ok) flags[0] = 1;
        }
        bar_sync_128(2);  // also: every read of xr / xc above is done
        if (!flags[0]) {
          ga = __ldcg(gp(n1, n1, ir, ic));
          gb = __ldcg(gp(n1, n1, ir, ic + 8));
        }
        xr[ir][ic] = pa;
        xr[ir][ic + 8] = pb;
        xc[ir][ic] = ga;
        xc[ir][ic + 8] = gb;
      }
    }
    __syncthreads();
    if (trace && tid == 0) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      unsigned long long *rec = trace + (size_t)s * 5;
      rec[0] = (unsigned long long)T_LT | ((unsigned long long)s << 8) |
               ((unsigned long long)(q < 0 ? 0 : q) << 24) | ((unsigned long long)s << 40);
      // SM id | SM cycles (saturated) of the solve, of the compute warps'
      // second phase, and of the whole step
      const unsigned long long ce = (unsigned long long)(clock64() - c0);
      rec[1] = (smid & 0xFFull) | (min((unsigned long long)(cx - c0), 0x3ffffull) << 8) |
               (min((unsigned long long)(cl - c1), 0x7ffffull) << 26) | (min(ce, 0x7ffffull) << 45);
      rec[2] = t0;
      rec[3] = t1;
      rec[4] = gtimer();
    }
    if (flags[1]) {
      // the first failure of the factor keeps its pivot (later diagonal
      // tiles, factored from skipped updates, may fail too)
      if (tid == 0 && atomicCAS(&st[ST_CODE], DEV_OK, DEV_NOTPD) == DEV_OK) st[ST_PIVOT] = gcol0 + s * PB + flags[1];
      return;
    }
    if (flags[0]) return;
  }
  // publish the last diagonal block
  if (io) {
    const int q = nbb - 1;
    if (ir >= ic) __stcg(gp(q, q, ir, ic), a[ir][ic]);
    if (ir >= ic + 8) __stcg(gp(q, q, ir, ic + 8), a[ir][ic + 8]);
    if (u < PB) __stcg(rinv_g + q * PB + u, rinv[u]);
    bar_sync_128(2);
    if (u == 0) {
      fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
      atomicExch(&state[q * nbb + q], q + 1);
    }
  }
}

// The chain of one tile on a cluster of three CTAs (ranks 0, 1 and 2 of
// cluster 0; the other clusters run the TRSM / UPD tasks).  The master (rank
// 0) keeps the four FP64 pipes of its SM for the leaf; the helpers do the
// rest of each step on their own SMs, and the three exchange data through
// distributed shared memory:
//   master, warps 0..3: factor C_s (block (s, s) after every panel < s, in
//     registers v0, v1) with the leaf, which leaves each scaled column
//     c_j / c_jj in xr[j] and 1/L_kk in rinv, released in groups (local
//     mbar[3], [7], [11], [13], [14], [15], [16]); then wait for C_{s+1}
//     (written into this CTA's xc, mbar[17]);
//   master, warps 4..7: two per helper forward alternate groups of columns,
//     then 1/L_kk; then they publish L_{s,s} and its pivot reciprocals;
//   first helper (rank 1), warps 0..3: block (s+1, s) after the panels < s-1
//     minus X_{s+1,s-1} X_{s,s-1}^T (X_{s+1,s-1} from the second helper's
//     step s-1), solved one column behind the leaf into X_{s+1,s}, scaled by
//     1/L_jj and published;
//   first helper, warps 4..7: X_{s+1,s} X_{s+1,s}^T accumulated over the
//     solve's columns 0..13 as the solve finishes each, sent negated into the
//     master's xc; columns 14 and 15 of the solve go to the master's xr as
//     soon as they are final, and the master adds their terms itself;
//   second helper (rank 2): block (s+2, s) solved the same way into
//     X_{s+2,s}, then panel s applied to block (s+2, s+2), the master's C'
//     of its step s+1 (into its lout; potrf_chain_helper2).
// The master's mbar phases advance once per step (parity s & 1).  flags[2]
// of each CTA is set by another when it stops (a failed pivot or wait), and
// every wait on a peer also gives up at that flag or the wait bound; the
// three CTAs end at one cluster barrier, so none leaves while another may
// still write into its shared memory.
__device__ __forceinline__ void potrf_chain_master(double *__restrict__ D, int nb, int gcol0, int *__restrict__ state,
                                                  double *__restrict__ rinv_g, int *st,
                                                  unsigned long long *__restrict__ trace, double (*lout)[PB + 1],
                                                  double (*mcol)[PB + 1], double (*xr)[PB + 1],
                                                  double (*xc)[PB + 1], double *rinv, double (*rinv2)[PB],
                                                  volatile int *flags, uint64_t *mbar) {
  const int nbb = nb / PB;
  const size_t ld = nb;
  const int tid = threadIdx.x, u = tid & 127;
  const bool io = tid >= 128;
  const int ir = u & (PB - 1), ic = u >> 4;                                 // warps 4..7
  const int i = u & (PB - 1), k0 = (u >> 5) + 4 * ((u >> 4) & 1), k1 = k0 + 8;  // warps 0..3
  auto gp = [&](int br, int bc, int r, int c) { return D + (size_t)(br * PB + r) + (size_t)(bc * PB + c) * ld; };
  // the helpers' objects (same layout: a helper's ms is the array this CTA
  // calls mcol; the second helper takes odd steps' columns in its a, which
  // this CTA calls lout)
  const uint32_t stop_h = peer_addr((const void *)&flags[2], 1), stop_h2 = peer_addr((const void *)&flags[2], 2);
  const uint32_t cfree_h2 = peer_addr(&mbar[34], 2);
  if (io) {
    xc[ir][ic] = __ldcg(gp(0, 0, ir, ic));
    xc[ir][ic + 8] = __ldcg(gp(0, 0, ir, ic + 8));
  }
  __syncthreads();
  double v0 = 0.0, v1 = 0.0;
  if (!io) {
    v0 = xc[i][k0];
    v1 = xc[i][k1];
  }
  for (int s = 0; s < nbb; s++) {
    const bool more = s + 1 < nbb;
    unsigned long long t0 = 0, t1 = 0;
    long long c0 = 0, c1 = 0, c7 = 0;  // trace only: SM cycles of the sub-phases
    if (trace && tid == 0) {
      t0 = gtimer();
      c0 = clock64();
    }
    if (!io) {
      // the scaled columns go to xr and mbar[0..16], from where warps 4..7
      // forward them
      // L_{s,s} is mcol[k][i] / sqrt(c_kk): lout stays free for C'
      const int fail = leaf16(u, v0, v1, mcol, nullptr, rinv, xr, mbar);
      if (fail && u == 0) flags[1] = fail;
      if (trace && tid == 0) {
        t1 = gtimer();
        c1 = clock64();
      }
      bar_arrive_256(6);  // the columns of L_{s,s} and 1/L_kk are in mcol and rinv
      if (more && !fail) {
        // C_{s+1} = C' - X_{s+1,s} X_{s+1,s}^T: the first helper sends -S,
        // S the sum over the solve's columns 0..13 (in xc; in step 0 block
        // (1, 1) minus S), the second helper C' = block (s+1, s+1) after
        // every panel < s (in lout, from step 1 on; released to it again
        // after the step's barrier), and the terms of columns 14 and 15
        // follow below
        if (!wait_from_peer(&mbar[17], (uint32_t)s & 1u, &flags[2])) {
          if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 4;
          flags[0] = 1;
        }
        if (trace && tid == 0) c7 = clock64();
        v0 = xc[i][k0];
        v1 = xc[i][k1];
        if (s >= 1) {
          if (!wait_from_peer(&mbar[18], (uint32_t)(s - 1) & 1u, &flags[2])) {
            if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 13;
            flags[0] = 1;
          }
          v0 += lout[i][k0];
          v1 += lout[i][k1];
        }
        // the terms of columns 14 and 15, u_j r_j u_j^T: the first helper's
        // u_j in xr rows 0, 1, the pivot reciprocals r_j in xr[j][PB]
        if (!wait_from_peer(&mbar[19], (uint32_t)s & 1u, &flags[2])) {
          if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 14;
          flags[0] = 1;
        }
        const double pa = xr[0][i] * xr[PB - 2][PB], pb = xr[1][i] * xr[PB - 1][PB];
        v0 = fma(-pa, xr[0][k0], v0);
        v1 = fma(-pa, xr[0][k1], v1);
        v0 = fma(-pb, xr[1][k0], v0);
        v1 = fma(-pb, xr[1][k1], v1);
      }
    } else {
      // forward the leaf's scaled columns, then 1/L_kk, to the helpers in
      // the groups the leaf releases them in (columns 0-3, 4-7, 8-11, 12-13,
      // 14, 15, then 1/L_kk: local mbar[3], [7], [11], [13], [14], [15],
      // [16]); each group's remote stores are released by one cluster-scope
      // arrival on that helper's barrier of the group's last column, and two
      // warps per helper take alternate groups, so that two releases are in
      // flight (the remote store and its release stay off the leaf's pivot
      // chain).  First helper (warps 4, 6): columns into its ms, 1/L_kk into
      // rinv2[s & 1] (barrier mbar[16] for even steps, mbar[35] for odd ones).
      // Second helper (warps 5, 7): even steps into its mcol and
      // mbar[0..16], odd ones into its lout and mbar[17..33], 1/L_kk into
      // rinv2[s & 1].
      const int fw = (tid >> 5) - 4, h = fw & 1, half = fw >> 1;
      if ((tid & 31) < PB && (h == 0 ? s + 1 < nbb : s + 2 < nbb)) {
        const uint32_t par = (uint32_t)s & 1u, odd = (uint32_t)s & 1u;
        const uint32_t rank = (uint32_t)h + 1u;
        const uint32_t ms_h = peer_addr(h == 1 && odd ? lout : mcol, rank);
        const uint32_t rinv_h = peer_addr(&rinv2[odd][0], rank);
        const uint32_t mbcol_h = peer_addr(&mbar[h == 1 && odd ? PB + 1 : 0], rank);
        const uint32_t mbr_h = peer_addr(&mbar[h == 0 ? (odd ? 35 : 16) : (odd ? 2 * PB + 1 : PB)], rank);
        const int l = tid & 31;  // < PB
#pragma unroll 1
        for (int g = half; g < 7; g += 2) {
          const int j0 = g < 3 ? 4 * g : (g == 3 ? 12 : g + 10);
          const int j1 = g < 3 ? 4 * g + 3 : (g == 3 ? 13 : g + 10);
          if (!wait_local(&mbar[j1], par, &flags[2])) {
            if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 7;
            flags[0] = 1;
          }
          for (int j = j0; j <= j1; j++) {
            if (j < PB) {
              st_peer_f64(ms_h + (uint32_t)(j * (PB + 1) + l) * 8u, xr[j][l]);
              if (l == j) st_peer_f64(ms_h + (uint32_t)(j * (PB + 1) + PB) * 8u, xr[j][PB]);
            } else {
              st_peer_f64(rinv_h + 8u * l, rinv[l]);
            }
          }
          // lane 0's cluster-scope release covers the stores its partners
          // ordered before it
          __syncwarp(0x0000ffffu);
          if (l == 0) arrive_peer(j1 < PB ? mbcol_h + 8u * j1 : mbr_h);
        }
      }
      bar_sync_256(6);
      if (!flags[1]) {
        // L_ik = c_ik / sqrt(c_kk), the diagonal c_kk / sqrt(c_kk)
        if (ir >= ic) __stcg(gp(s, s, ir, ic), mcol[ic][ir] * rinv[ic]);
        if (ir >= ic + 8) __stcg(gp(s, s, ir, ic + 8), mcol[ic + 8][ir] * rinv[ic + 8]);
        if (u < PB) __stcg(rinv_g + s * PB + u, rinv[u]);
        bar_sync_128(2);
        if (u == 0) {
          fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
          atomicExch(&state[s * nbb + s], s + 1);
        }
      }
    }
    // one decision for all threads: a peer may set flags[2] at any time
    const bool stop = __syncthreads_or(flags[1] | flags[0] | flags[2]) != 0;
    // C' in lout is read: the second helper's next one may come (released by
    // an I/O thread, off the compute warps' way to the next leaf)
    if (tid == 128 && !stop && s >= 1 && s + 2 < nbb) arrive_peer(cfree_h2);
    if (trace && tid == 0) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      unsigned long long *rec = trace + (size_t)s * 5;
      rec[0] = (unsigned long long)T_LT | ((unsigned long long)s << 8) |
               ((unsigned long long)(s > 0 ? s - 1 : 0) << 24) | ((unsigned long long)s << 40);
      // SM id | SM cycles (saturated) of the leaf, of the wait for X_{s+1,s}
      // after it, and of the whole step
      const unsigned long long ce = (unsigned long long)(clock64() - c0);
      rec[1] = (smid & 0xFFull) | (min((unsigned long long)(c1 - c0), 0x3ffffull) << 8) |
               (min((unsigned long long)(c7 > c1 ? c7 - c1 : 0), 0x7ffffull) << 26) | (min(ce, 0x7ffffull) << 45);
      rec[2] = t0;
      rec[3] = t1;
      rec[4] = gtimer();
    }
    if (stop) {
      if (tid == 0) {
        // the first failure of the factor keeps its pivot
        if (flags[1] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_NOTPD) == DEV_OK) st[ST_PIVOT] = gcol0 + s * PB + flags[1];
        st_peer_s32(stop_h, 1);
        st_peer_s32(stop_h2, 1);
      }
      break;
    }
  }
  cluster_barrier();
}

__device__ __forceinline__ void potrf_chain_helper1(double *__restrict__ D, int nb, int *__restrict__ state, int *st,
                                                  unsigned long long *__restrict__ trace, double (*ms)[PB + 1],
                                                  double (*xprev)[PB + 1], double (*xo)[PB + 1],
                                                  double (*uu)[PB + 1], double (*rinv2)[PB], volatile int *flags,
                                                  uint64_t *mbar) {
  const int nbb = nb / PB;
  const size_t ld = nb;
  const int tid = threadIdx.x, u = tid & 127;
  const bool cw = tid < 128;                        // warps 0..3: B and the solve; 4..7: C'
  const int cr = u >> 4, ct = u & (PB - 1);         // warps 0..3: rows cr, cr + 8 of column ct
  const int ir = u & (PB - 1), ic = u >> 4;         // warps 4..7: entries (ir, ic), (ir, ic + 8)
  auto gp = [&](int br, int bc, int r, int c) { return D + (size_t)(br * PB + r) + (size_t)(bc * PB + c) * ld; };
  // the master's objects: C_{s+1} goes to its xc (this CTA's xo at the same
  // address); its mbar[17] counts one arrival per warp of this CTA
  const uint32_t xc_m = peer_addr(xo, 0), xr_m = peer_addr(xprev, 0);  // the master's xc and xr
  const uint32_t mbx_m = peer_addr(&mbar[17], 0), stop_m = peer_addr((const void *)&flags[2], 0);
  const uint32_t mbu_m = peer_addr(&mbar[19], 0);
  const uint32_t stop_h2 = peer_addr((const void *)&flags[2], 2);
  for (int s = 0; s + 1 < nbb; s++) {
    const int n1 = s + 1;
    const uint32_t par = (uint32_t)s & 1u;
    unsigned long long t0 = 0, t1 = 0, t2 = 0;  // trace only
    // block (n1, s) after the panels < s-1 (UPD tasks, usually complete long
    // before) and X_{n1,s-1} (the second helper's step s-1)
    if (tid == 0) {
      if (trace) t0 = gtimer();
      if (!dag_wait2(state, n1 * nbb + s, s - 1, s >= 1 ? n1 * nbb + (s - 1) : -1, s, st)) flags[0] = 1;
      fence_acq_rel_gpu();
      if (trace) t1 = gtimer();
    }
    if (__syncthreads_or(flags[0] | flags[2])) break;
    double va = 0.0, vb = 0.0;
    if (cw) {
      va = __ldcg(gp(n1, s, cr, ct));
      vb = __ldcg(gp(n1, s, cr + 8, ct));
    } else if (s >= 1) {
      xo[ir][ic] = __ldcg(gp(n1, s - 1, ir, ic));
      xo[ir][ic + 8] = __ldcg(gp(n1, s - 1, ir, ic + 8));
    }
    if (s >= 1) {
      __syncthreads();  // X_{n1,s-1} is in xo
      // panel s-1 applied to block (n1, s): B -= X_{n1,s-1} X_{s,s-1}^T
      if (cw) {
        va -= panel_dot(xo, xprev, cr, ct);
        vb -= panel_dot(xo, xprev, cr + 8, ct);
      }
    }
    if (cw) {
      // X_{n1,s} L_{s,s}^T = B, column j as soon as the master's leaf has
      // formed column j of L_{s,s} (in the unscaled form x_j L_jj)
#pragma unroll
      for (int j = 0; j < PB; j++) {
        if (j >= PB - 2) {
          // u_{.,j} is final once column j-1 is applied: the last two go to
          // the master (rows 0, 1 of its xr, forwarded long before), which
          // subtracts their terms of X X^T itself
          if (ct == j) {
            st_peer_f64(xr_m + (uint32_t)((j - (PB - 2)) * (PB + 1) + cr) * 8u, va);
            st_peer_f64(xr_m + (uint32_t)((j - (PB - 2)) * (PB + 1) + cr + 8) * 8u, vb);
          }
          __syncwarp();
          if ((tid & 31) == 0) arrive_peer(mbu_m);
        }
        if (col_group_first(j) && !wait_from_peer(&mbar[col_group_bar(j)], par, &flags[2])) {
          if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 5;
          flags[0] = 1;
        }
        if (j < PB - 2 && ct == j) {
          // u_{cr,j}, u_{cr+8,j} are final: to the accumulation (warps 4..7)
          uu[j][cr] = va;
          uu[j][cr + 8] = vb;
          tc::mbar_arrive(&mbar[18 + j]);
        }
        const double aj = __shfl_sync(0xffffffffu, va, j, PB), bj = __shfl_sync(0xffffffffu, vb, j, PB);
        if (ct > j) {
          const double mj = ms[j][ct];
          va = fma(-aj, mj, va);
          vb = fma(-bj, mj, vb);
        }
      }
      if (trace && tid == 0) t2 = gtimer();
    } else {
      // S = X X^T needs no square root: with u_j = x_j L_jj (the solve's
      // unscaled columns) and r_j = 1/c_jj = 1/L_jj^2, S = sum_j u_j r_j
      // u_j^T, accumulated column by column as the solve finishes each one.
      // The master adds C' (block (n1, n1) after every panel < s, from the
      // second helper) to -S; in step 0, C' is block (1, 1) itself, and it
      // goes in here.
      if (s == 0) {
        va = __ldcg(gp(n1, n1, ir, ic));
        vb = __ldcg(gp(n1, n1, ir, ic + 8));
      }
      // p = r_j u_{ir,j} is formed as column j arrives and used two steps of
      // the loop later, and even and odd columns go to two sums, so that no
      // FMA waits for the multiply or the FMA before it; the odd sum joins the
      // even one before the last two columns' FMAs
      // (columns 0..PB-3; the master takes the last two)
      double va1 = 0.0, vb1 = 0.0;
      double p1 = 0.0, q10 = 0.0, q11 = 0.0;  // column j - 1
      double p2 = 0.0, q20 = 0.0, q21 = 0.0;  // column j - 2
#pragma unroll 2
      for (int j = 0; j < PB - 2; j++) {
        if (j >= 2) {
          if (j & 1) {
            va1 = fma(-p2, q20, va1);  // column j - 2, odd
            vb1 = fma(-p2, q21, vb1);
          } else {
            va = fma(-p2, q20, va);
            vb = fma(-p2, q21, vb);
          }
        }
        p2 = p1;
        q20 = q10;
        q21 = q11;
        if (!wait_local(&mbar[18 + j], par, &flags[2])) {  // arrivals of warps 0..3 of this CTA
          if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 8;
          flags[0] = 1;
        }
        p1 = uu[j][ir] * ms[j][PB];
        q10 = uu[j][ic];
        q11 = uu[j][ic + 8];
      }
      va += va1;
      vb += vb1;
      va = fma(-p2, q20, va);  // column PB - 4
      vb = fma(-p2, q21, vb);
      va = fma(-p1, q10, va);  // column PB - 3
      vb = fma(-p1, q11, vb);
      // -S (step 0: C_1) entries (ir, ic), (ir, ic + 8) into the master's xc:
      // its next leaf starts from C' - S
      st_peer_f64(xc_m + (uint32_t)(ir * (PB + 1) + ic) * 8u, va);
      st_peer_f64(xc_m + (uint32_t)(ir * (PB + 1) + ic + 8) * 8u, vb);
      __syncwarp();
      if ((tid & 31) == 0) arrive_peer(mbx_m);  // one per warp (warps 4..7)
    }
    // X_{n1,s} = u / L_jj, for TRSM tasks and the next step's B.  1/L_jj
    // comes in rinv2[s & 1] (barrier mbar[16] for even steps, mbar[35] for
    // odd ones, a phase every other step): the master may reach the end of
    // its next leaf before this wait
    if (cw && !wait_from_peer(&mbar[(s & 1) ? 35 : 16], (uint32_t)(s >> 1) & 1u, &flags[2])) {
      if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 6;
      flags[0] = 1;
    }
    if (__syncthreads_or(flags[0] | flags[2])) break;  // every read of xo and xprev above is done
    if (cw) {
      const double xa = va * rinv2[s & 1][ct], xb = vb * rinv2[s & 1][ct];
      xprev[cr][ct] = xa;
      xprev[cr + 8][ct] = xb;
      __stcg(gp(n1, s, cr, ct), xa);
      __stcg(gp(n1, s, cr + 8, ct), xb);
    }
    if (cw) {
      // publish X_{n1,s}
      bar_sync_128(2);
      if (tid == 0) {
        fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
        atomicExch(&state[n1 * nbb + s], s + 1);
        if (trace) {
          unsigned smid;
          asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
          unsigned long long *rec = trace + (size_t)s * 5;
          rec[0] = (unsigned long long)T_HELP | ((unsigned long long)n1 << 8) | ((unsigned long long)s << 24) |
                   ((unsigned long long)s << 40);
          // SM id | ns from the inputs to the end of the solve (saturated)
          rec[1] = (smid & 0xFFull) | (min(t2 - t1, 0x3ffffull) << 8);
          rec[2] = t0;
          rec[3] = t1;
          rec[4] = gtimer();  // C sent, X published
        }
      }
    }
    __syncthreads();
  }
  // a stop of this CTA (failed wait) stops the other two CTAs' waits as well
  if (tid == 0 && flags[0]) {
    st_peer_s32(stop_m, 1);
    st_peer_s32(stop_h2, 1);
  }
  cluster_barrier();
}

// The chain's second helper (CTA rank 2): in step s it solves block (s+2, s)
// one column behind the master's leaf, as the first helper solves block
// (s+1, s), and publishes X_{s+2,s}, which the first helper's step s+1 and
// the UPD tasks of panel s read.  The block's update by panel s-1,
// D = X_{s+2,s-1} X_{s,s-1}^T, waits for X_{s+2,s-1} from a TRSM task, which
// comes late in the step; the solve is linear, so warps 0..3 solve block
// (s+2, s) after the panels < s-1 (UPD tasks, ready early) column by column
// with the leaf, warps 4..7 form D once its inputs are published and solve
// it against the columns received so far, and X_{s+2,s} is the difference.
// It applies panel s to block (s+2, s+2) (UPD(s+2, s+2, s)) early in its
// next step, on warps 0..3 before their solve: C' of the master's step s+1,
// which adds it to the first helper's -S.
// The columns come in two buffers (ms0 and barriers mbar[0..16] in even
// steps, ms1 and mbar[17..33] in odd ones, 1/L_kk in rinv2[s & 1]), so that
// the master may run a step ahead of this CTA: its step s+2 waits for the
// first helper's step s+1, which waits for this CTA's X_{s+2,s}.
__device__ __forceinline__ void potrf_chain_helper2(double *__restrict__ D, int nb, int *__restrict__ state, int *st,
                                                 unsigned long long *__restrict__ trace, double (*ms0)[PB + 1],
                                                 double (*ms1)[PB + 1], double (*xn)[PB + 1], double (*xs)[PB + 1],
                                                 double (*rinv2)[PB], volatile int *flags, uint64_t *mbar) {
  const int nbb = nb / PB;
  const size_t ld = nb;
  const int tid = threadIdx.x, u = tid & 127;
  const bool cw = tid < 128;                 // warps 0..3: the block; 4..7: D
  const int cr = u >> 4, ct = u & (PB - 1);  // rows cr, cr + 8 of column ct
  auto gp = [&](int br, int bc, int r, int c) { return D + (size_t)(br * PB + r) + (size_t)(bc * PB + c) * ld; };
  const uint32_t stop_m = peer_addr((const void *)&flags[2], 0), stop_h = peer_addr((const void *)&flags[2], 1);
  const uint32_t cp_m = peer_addr(ms1, 0), cready_m = peer_addr(&mbar[18], 0);  // the master's lout is its a
  // Hand-over k, by warps 0..3: panel k applied to block (k+2, k+2) (after
  // the panels < k, UPD tasks), with X_{k+2,k} in xn: C' of the master's step
  // k+1, written into its lout once it has read hand-over k-1 there (this
  // CTA's mbar[34]) and released by one arrival per warp on its mbar[18].
  auto hand_over = [&](int k) {
    const int nk = k + 2;
    if (tid == 0) {
      if (!dag_wait(state, nk * nbb + nk, k, st)) flags[0] = 1;
      fence_acq_rel_gpu();
    }
    bar_sync_128(2);
    const double c0 = __ldcg(gp(nk, nk, cr, ct)) - panel_dot(xn, xn, cr, ct);
    const double c1 = __ldcg(gp(nk, nk, cr + 8, ct)) - panel_dot(xn, xn, cr + 8, ct);
    if (k >= 1 && !wait_from_peer(&mbar[34], (uint32_t)(k - 1) & 1u, &flags[2])) {
      if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 12;
      flags[0] = 1;
    }
    st_peer_f64(cp_m + (uint32_t)(cr * (PB + 1) + ct) * 8u, c0);
    st_peer_f64(cp_m + (uint32_t)((cr + 8) * (PB + 1) + ct) * 8u, c1);
    __syncwarp();
    if ((tid & 31) == 0) arrive_peer(cready_m);
  };
  for (int s = 0; s + 2 < nbb; s++) {
    const int n2 = s + 2, b = s & 1;
    const uint32_t par = (uint32_t)(s >> 1) & 1u;
    double(*ms)[PB + 1] = b ? ms1 : ms0;
    uint64_t *mb = mbar + (b ? PB + 1 : 0);
    unsigned long long t0 = 0, t1 = 0, t2 = 0;  // trace only
    if (tid == 0) {
      if (trace) t0 = gtimer();
      // block (s+2, s) after the panels < s-1
      if (!dag_wait(state, n2 * nbb + s, s - 1, st)) flags[0] = 1;
      fence_acq_rel_gpu();
    }
    if (__syncthreads_or(flags[0] | flags[2])) break;
    double va = 0.0, vb = 0.0;
    if (cw) {
      // first the previous step's hand-over (its X is in xn; the leaf's first
      // columns arrive meanwhile and the solve below catches up), then the
      // block after the panels < s-1
      if (s >= 1) {
        hand_over(s - 1);
        bar_arrive_256(4);  // xn may take D's solve
      }
      va = __ldcg(gp(n2, s, cr, ct));
      vb = __ldcg(gp(n2, s, cr + 8, ct));
    } else if (s >= 1) {
      // X_{s+2,s-1} (TRSM task) and X_{s,s-1} (the first helper), then D; the
      // rows of X_{s+2,s-1} come from global memory (xn holds X_{s+1,s-1} for
      // the hand-over)
      if (tid == 128) {
        if (!dag_wait2(state, n2 * nbb + (s - 1), s, s * nbb + (s - 1), s, st)) flags[0] = 1;
        fence_acq_rel_gpu();
        // trace: the arrival time, for thread 0, in xs's padding column
        if (trace) xs[0][PB] = __longlong_as_double((long long)gtimer());
      }
      bar_sync_128(3);
      xs[cr][ct] = __ldcg(gp(s, s - 1, cr, ct));
      xs[cr + 8][ct] = __ldcg(gp(s, s - 1, cr + 8, ct));
      bar_sync_128(3);
      double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
#pragma unroll 4
      for (int k = 0; k < PB; k += 2) {
        a0 = fma(__ldcg(gp(n2, s - 1, cr, k)), xs[ct][k], a0);
        b0 = fma(__ldcg(gp(n2, s - 1, cr + 8, k)), xs[ct][k], b0);
        a1 = fma(__ldcg(gp(n2, s - 1, cr, k + 1)), xs[ct][k + 1], a1);
        b1 = fma(__ldcg(gp(n2, s - 1, cr + 8, k + 1)), xs[ct][k + 1], b1);
      }
      va = a0 + a1;
      vb = b0 + b1;
    }
    // both halves: the unscaled solve of their 16 x 16 block against L_{s,s}
    // (warps 4..7 only when there is a D), column j once the leaf has formed
    // column j (in the unscaled form x_j L_jj)
    if (cw || s >= 1) {
#pragma unroll
      for (int j = 0; j < PB; j++) {
        if (col_group_first(j) && !wait_from_peer(&mb[col_group_bar(j)], par, &flags[2])) {
          if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 9;
          flags[0] = 1;
        }
        const double aj = __shfl_sync(0xffffffffu, va, j, PB), bj = __shfl_sync(0xffffffffu, vb, j, PB);
        if (ct > j) {
          const double mj = ms[j][ct];
          va = fma(-aj, mj, va);
          vb = fma(-bj, mj, vb);
        }
      }
    }
    if (!cw && s >= 1) {
      bar_sync_256(4);  // warps 0..3 have read xn (the hand-over)
      xn[cr][ct] = va;
      xn[cr + 8][ct] = vb;
    }
    if (cw && !wait_from_peer(&mb[PB], par, &flags[2])) {
      if (!flags[2] && atomicCAS(&st[ST_CODE], DEV_OK, DEV_TIMEOUT) == DEV_OK) st[ST_AUX] = 10;
      flags[0] = 1;
    }
    if (__syncthreads_or(flags[0] | flags[2])) break;  // D's solve is in xn
    if (cw) {
      if (trace && tid == 0) {
        t2 = gtimer();
        t1 = s >= 1 ? (unsigned long long)__double_as_longlong(xs[0][PB]) : t0;
      }
      if (s >= 1) {
        va -= xn[cr][ct];
        vb -= xn[cr + 8][ct];
      }
      const double r = rinv2[b][ct];
      va *= r;
      vb *= r;
      __stcg(gp(n2, s, cr, ct), va);
      __stcg(gp(n2, s, cr + 8, ct), vb);
      xn[cr][ct] = va;  // for hand-over s; each thread overwrites the entries of D's solve it read
      xn[cr + 8][ct] = vb;
      bar_sync_128(2);
      if (tid == 0) {
        fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
        atomicExch(&state[n2 * nbb + s], s + 1);
        if (trace) {
          unsigned smid;
          asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
          unsigned long long *rec = trace + (size_t)s * 5;
          rec[0] = (unsigned long long)T_HELP2 | ((unsigned long long)n2 << 8) | ((unsigned long long)s << 24) |
                   ((unsigned long long)s << 40);
          // SM id | ns from the arrival of D's inputs to the end of both solves
          rec[1] = (smid & 0xFFull) | (min(t2 - t1, 0x3ffffull) << 8);
          rec[2] = t0;
          rec[3] = t1;
          rec[4] = gtimer();
        }
      }
    }
    __syncthreads();  // xn holds X_{s+2,s}
  }
  // the last hand-over, unless the chain has stopped (one decision for all)
  if (!__syncthreads_or(flags[0] | flags[2]) && cw && nbb >= 3) hand_over(nbb - 3);
  if (tid == 0 && flags[0]) {
    st_peer_s32(stop_m, 1);
    st_peer_s32(stop_h, 1);
  }
  cluster_barrier();
}

// One tile: at most 64 registers per thread (4 CTAs of 256 threads per SM),
// because it shares every SM with the persistent bulk GEMM of the mixed
// factor and a larger register footprint measurably slowed both.  The batch
// form runs alone.
template <bool BATCH>
__global__ void __launch_bounds__(PB * PB, BATCH ? 1 : 4)
    k_potrf_dag(double *__restrict__ D0, int nb, int gcol0, const short4 *__restrict__ tasks, int ntasks,
                int *__restrict__ ws, double *__restrict__ rinv_all, int *st,
                unsigned long long *__restrict__ trace, const long *__restrict__ dtiles, int nbat,
                int *__restrict__ bad_out) {
  __shared__ double a[PB][PB + 1];   // L of the block solved against, then the block factored
  __shared__ double m[PB][PB + 1];   // L scaled by the pivot reciprocals (solves)
  __shared__ double xr[PB][PB + 1];  // panel rows of block r
  __shared__ double xc[PB][PB + 1];  // panel rows of block c (or s)
  __shared__ double rinv[PB];
  __shared__ double rinv2[2][PB];         // the cluster form's helpers: 1/L_kk of even / odd steps
  __shared__ int s_task, s_ok, bad, s_leave;
  __shared__ int mflags[3];
  __shared__ uint64_t mbar[2 * PB + 4];  // the cluster form's hand-over barriers
  // ws = {task counter, then state[nbb*nbb] per tile, then (single tile) the
  // master's SM id + 1 and the number of CTAs that left it}; rinv_all = nb
  // pivot reciprocals per tile.  A batch of nbat tiles (dtiles = their
  // indices in D0) interleaves the tiles' task lists: task t is task t / nbat
  // of tile t % nbat, so each tile's tasks stay in topological order.
  int *counter = ws;
  const int nbb = nb / PB;
  const int tx = threadIdx.x % PB, ty = threadIdx.x / PB;
  const size_t ld = nb;
  // Single tile: a CTA on one of the chain's SMs fetches no task (from its
  // start if it starts there after the chain, else from its next fetch).  On
  // the master's SM it stays resident and idle until the chain has published
  // its last diagonal block, so that neither it nor a CTA of another kernel
  // takes that SM's FP64 pipes from the leaf; a CTA that left instead was
  // replaced there by the launch's next pending CTA, and once the number that
  // could leave was used up, the rest worked there.  At most kMaxIdle CTAs
  // idle.  On a helper's SM it leaves (at most half the launch leaves, so the
  // chain always keeps workers): idle CTAs there measurably slowed the
  // helpers' steps.
  // ws extras: master SM id + 1, idle CTAs, the helpers' SM ids + 1, CTAs
  // that left
  constexpr int kMaxIdle = 12;
  int *master_sm = ws + 1 + (size_t)nbat * nbb * nbb;
  unsigned my_sm = 0;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(my_sm));
  // Cluster form (one tile launched as clusters of three): cluster 0 runs
  // the chain (rank 0 the master, ranks 1 and 2 the helpers) and never
  // fetches a task; the other CTAs fetch tasks 1, 2, ...  Cluster 0 always
  // reaches its final cluster barrier: its loops stop on the status word
  // inside their bounded waits rather than returning here.
  const bool clus = !BATCH && cluster_nctarank() == 3;
  if (clus && cluster_id_x() == 0) {
    const uint32_t rank = cluster_ctarank();
    if (threadIdx.x == 0) {
      mflags[0] = mflags[1] = mflags[2] = 0;
      if (rank == 0) {
        // per column / rinv: the 16 leaf threads; mbar[17]: C from the first
        // helper's warps 4..7
        for (int j = 0; j <= PB; j++) tc::mbar_init(&mbar[j], PB);
        tc::mbar_init(&mbar[17], 4);
        tc::mbar_init(&mbar[18], 4);  // C' from the second helper: one arrival per warp 4..7 of it
        tc::mbar_init(&mbar[19], 8);  // u_14, u_15 from the first helper: one arrival per warp 0..3 and column
      } else if (rank == 1) {
        // columns (one arrival of the master's forwarding warp), rinv of even
        // / odd steps, column j of u (one thread per half-warp of warps 0..3)
        for (int j = 0; j <= PB; j++) tc::mbar_init(&mbar[j], 1);
        tc::mbar_init(&mbar[35], 1);
        for (int j = 0; j < PB; j++) tc::mbar_init(&mbar[18 + j], 8);
      } else {
        // columns and rinv of even / odd steps; mbar[34]: the master has read
        // the last C' (one arrival)
        for (int j = 0; j < 2 * (PB + 1); j++) tc::mbar_init(&mbar[j], 1);
        tc::mbar_init(&mbar[34], 1);
      }
      tc::fence_barrier_init();
      atomicExch(master_sm + (rank == 0 ? 0 : rank + 1), (int)my_sm + 1);
    }
    cluster_barrier();  // the three CTAs' barriers exist before any remote access
    double *rinv_g = rinv_all;
    unsigned long long *tr = trace ? trace + (size_t)(ntasks + (size_t)rank * nbb) * 5 : nullptr;
    if (rank == 0)
      potrf_chain_master(D0, nb, gcol0, ws + 1, rinv_g, st, tr, a, m, xr, xc, rinv, rinv2, mflags, mbar);
    else if (rank == 1)
      potrf_chain_helper1(D0, nb, ws + 1, st, tr, m, xr, xc, a, rinv2, mflags, mbar);
    else
      potrf_chain_helper2(D0, nb, ws + 1, st, tr, m, a, xr, xc, rinv2, mflags, mbar);
    return;
  }
  // a factor that has already failed (status set by an earlier launch) stops
  if (*((volatile const int *)st) != DEV_OK) return;
  if (threadIdx.x == 0) s_leave = 0;
  while (true) {
    if (threadIdx.x == 0) {
      if (!s_leave && !BATCH) {
        const int me = (int)my_sm + 1;
        if (*((volatile int *)master_sm) == me) {
          if (atomicAdd(master_sm + 1, 1) < kMaxIdle) s_leave = 2;
        } else if ((*((volatile int *)(master_sm + 2)) == me || *((volatile int *)(master_sm + 3)) == me) &&
                   atomicAdd(master_sm + 4, 1) < (int)gridDim.x / 2) {
          s_leave = 1;
        }
      }
      s_task = s_leave ? INT_MAX : atomicAdd(counter, 1) + (clus ? 1 : 0);  // cluster form: task 0 is cluster 0's
      if (s_leave == 2) idle_until(ws + 1 + (size_t)(nbb - 1) * (nbb + 1), nbb, st);  // L of the last diagonal block
    }
    __syncthreads();
    int t = s_task;
    // one tile (the single-matrix factor) compiles without the batch indexing
    const int bt = BATCH ? t % nbat : 0;
    if (t >= (BATCH ? ntasks * nbat : ntasks)) return;
    double *D = BATCH ? D0 + (size_t)dtiles[bt] * nb * nb : D0;
    int *state = BATCH ? ws + 1 + (size_t)bt * nbb * nbb : ws + 1;
    double *rinv_g = BATCH ? rinv_all + (size_t)bt * nb : rinv_all;
    auto blk = [&](int br, int bc) { return D + (size_t)(br * PB + ty) + (size_t)(bc * PB + tx) * ld; };
    short4 tk = tasks[BATCH ? t / nbat : t];
    int kind = tk.x, r = tk.y, c = tk.z, s = tk.w;  // LT: (s, s-1, s); TRSM: (r, s, s); UPD: (r, c, s)
    if (!BATCH && kind == T_MASTER) {
      if (threadIdx.x == 0) atomicExch(master_sm, (int)my_sm + 1);
      potrf_master(D, nb, gcol0, state, rinv_g, st, trace ? trace + (size_t)ntasks * 5 : nullptr, a, m, xr, xc, rinv,
                   mflags);
      return;
    }
    unsigned long long t_fetch = 0;
    if (trace && threadIdx.x == 0) t_fetch = gtimer();
    if (threadIdx.x == 0) {
      bool ok;
      if (BATCH && kind == T_LT)
        // first the inputs other tasks produce (usually ready long before
        // LT(s-1) ends): X_{s,s-2}, block (s,s-1) and the diagonal block
        ok = dag_wait3(state, s >= 2 ? s * nbb + (s - 2) : -1, s - 1, s >= 1 ? s * nbb + (s - 1) : -1, s - 2,
                       s * nbb + s, s - 1, st);
      else if (kind == T_TRSM)
        // the inputs of the panel s-1 update first; L_{s,s} is awaited below
        ok = dag_wait3(state, s >= 1 ? r * nbb + (s - 1) : -1, s, s >= 1 ? s * nbb + (s - 1) : -1, s,
                       r * nbb + s, s - 1, st);
      else
        ok = dag_wait3(state, r * nbb + s, s + 1, c * nbb + s, s + 1, r * nbb + c, s, st);
      fence_acq_rel_gpu();
      s_ok = ok;
      bad = 0;
      if (trace) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        unsigned long long *rec = trace + (size_t)t * 5;
        rec[0] = (unsigned long long)kind | ((unsigned long long)r << 8) | ((unsigned long long)c << 24) |
                 ((unsigned long long)s << 40);
        rec[1] = smid;
        rec[2] = t_fetch;
        rec[3] = gtimer();
      }
    }
    __syncthreads();
    if (!s_ok) return;
    if (kind == T_UPD) {
      xr[ty][tx] = __ldcg(blk(r, s));
      xc[ty][tx] = __ldcg(blk(c, s));
      double *cp = blk(r, c);
      double v = __ldcg(cp);
      __syncthreads();
      __stcg(cp, v - panel_dot(xr, xc, ty, tx));
    } else if (kind == T_TRSM) {
      // Solve block (r, s) against L_{s,s} after its fused update by panel
      // s-1, which runs as soon as X_{s,s-1} is published, before L_{s,s}
      // (the chain publishes X_{s,s-1} before it factors block (s, s)).  Row
      // ty's 16 lanes exchange entries by shuffle.
      double *bp = blk(r, s);
      double v = __ldcg(bp);
      if (s >= 1) {
        xr[ty][tx] = __ldcg(blk(r, s - 1));
        xc[ty][tx] = __ldcg(blk(s, s - 1));
        __syncthreads();
        v -= panel_dot(xr, xc, ty, tx);
      }
      if (threadIdx.x == 0) {
        s_ok = dag_wait(state, s * nbb + s, s + 1, st);  // L_{s,s}
        fence_acq_rel_gpu();
      }
      __syncthreads();
      if (!s_ok) return;
      a[ty][tx] = __ldcg(blk(s, s));
      if (threadIdx.x < PB) rinv[threadIdx.x] = __ldcg(rinv_g + s * PB + threadIdx.x);
      __syncthreads();
      m[ty][tx] = a[ty][tx] * rinv[tx];
      __syncthreads();
#pragma unroll
      for (int j = 0; j < PB; j++) {
        double vj = __shfl_sync(0xffffffffu, v, j, PB);
        if (tx > j) v = fma(-vj, m[tx][j], v);
      }
      __stcg(bp, v * rinv[tx]);
    } else if (BATCH) {
      // LT(s) (batch form; one tile runs the chain in potrf_master): the
      // inputs other tasks produce are loaded first; block (s, s-1)
      // gets its fused update by panel s-2 as soon as LT(s-1) has published
      // X_{s-1,s-2}; once LT(s-1) has ended it is solved against L_{s-1,s-1},
      // published, applied to the diagonal block, and the diagonal block is
      // factored.
      const int q = s - 1;
      double *bp = blk(s, q >= 0 ? q : 0);
      const double dg = __ldcg(blk(s, s));
      double v = 0.0;
      if (q >= 0) {
        v = __ldcg(bp);
        if (q >= 1) xr[ty][tx] = __ldcg(blk(s, q - 1));
      }
      if (q >= 1) {
        if (threadIdx.x == 0) {
          s_ok = dag_wait(state, q * nbb + (q - 1), q, st);  // X_{q,q-1} published
          fence_acq_rel_gpu();
        }
        __syncthreads();
        if (!s_ok) return;
        xc[ty][tx] = __ldcg(blk(q, q - 1));
        __syncthreads();
        v -= panel_dot(xr, xc, ty, tx);
      }
      if (q >= 0) {
        if (threadIdx.x == 0) {
          s_ok = dag_wait(state, q * nbb + q, s, st);  // LT(s-1) has ended
          fence_acq_rel_gpu();
        }
        __syncthreads();  // also orders the reads of xr / xc above before their reuse
        if (!s_ok) return;
        a[ty][tx] = __ldcg(blk(q, q));
        if (threadIdx.x < PB) rinv[threadIdx.x] = __ldcg(rinv_g + q * PB + threadIdx.x);
        __syncthreads();
        m[ty][tx] = a[ty][tx] * rinv[tx];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PB; j++) {
          double vj = __shfl_sync(0xffffffffu, v, j, PB);
          if (tx > j) v = fma(-vj, m[tx][j], v);
        }
        xr[ty][tx] = v * rinv[tx];  // X_{s,q}
      }
      xc[ty][tx] = dg;
      __syncthreads();
      if (threadIdx.x >= 128) {
        // warps 4..7 publish X_{s,q} (lanes along columns of the block)
        if (q >= 0) {
          const int e = threadIdx.x - 128, rr = e & (PB - 1), cc = e >> 4;
          double *xp = D + (size_t)(s * PB + rr) + (size_t)(q * PB + cc) * ld;
          __stcg(xp, xr[rr][cc]);
          __stcg(xp + 8 * ld, xr[rr][cc + 8]);
          bar_sync_128(2);
          if (threadIdx.x == 128) {
            fence_acq_rel_gpu();  // releases the stores ordered before it by the barrier
            atomicExch(&state[s * nbb + q], s);
          }
        }
      } else {
        // warps 0..3: the diagonal block minus X X^T, then the leaf
        const int u = threadIdx.x, i = u & (PB - 1);
        const int k0 = (u >> 5) + 4 * ((u >> 4) & 1), k1 = k0 + 8;
        double v0 = xc[i][k0], v1 = xc[i][k1];
        if (q >= 0) {
          v0 -= panel_dot(xr, xr, i, k0);
          v1 -= panel_dot(xr, xr, i, k1);
        }
        const int fail = leaf16(u, v0, v1, m, a, rinv);
        if (fail && u == 0) bad = fail;
      }
      __syncthreads();
      if (bad) {
        if (threadIdx.x == 0) {
          if (bad_out) {
            // the batch goes on: only this matrix is flagged, with its first
            // non-positive pivot column (its factor is not used)
            atomicCAS(&bad_out[bt], 0, gcol0 + s * PB + bad);
          } else if (atomicCAS(&st[ST_CODE], DEV_OK, DEV_NOTPD) == DEV_OK) {
            st[ST_PIVOT] = gcol0 + s * PB + bad;
            st[ST_AUX] = bt;  // which tile of the batch
          }
        }
        if (!bad_out) return;
      }
      if (ty >= tx) __stcg(blk(s, s), a[ty][tx]);
      if (threadIdx.x < PB) __stcg(rinv_g + s * PB + threadIdx.x, rinv[threadIdx.x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_acq_rel_gpu();
      if (BATCH && kind == T_LT) {
        atomicExch(&state[s * nbb + s], s + 1);  // X_{s,s-1} was published before the leaf
      } else {
        atomicExch(&state[r * nbb + c], s + 1);
      }
      if (trace) trace[(size_t)t * 5 + 4] = gtimer();
    }
  }
}

// Task list of the dataflow POTRF for nbb blocks per side (see k_potrf_dag),
// in topological, lookahead-first order.  With master = true the LT tasks
// are replaced by one T_MASTER task at the head of the list (single tile);
// clus = true: the chain runs on a cluster of three CTAs.
static void dag_tasks(int nbb, std::vector<short4> &out, bool master, bool clus = false) {
  out.clear();
  auto push = [&](int kind, int r, int c, int s) {
    out.push_back(make_short4((short)kind, (short)r, (short)c, (short)s));
  };
  if (master)
    push(T_MASTER, 0, 0, 0);
  else
    push(T_LT, 0, 0, 0);
  // Cluster form: the helpers solve blocks (c+1, c) and (c+2, c) of each
  // column c, so TRSM(c+2, c) is not listed either.
  for (int r = 2; r < nbb; r++)
    if (!clus || r != 2) push(T_TRSM, r, 0, 0);
  for (int s = 0; s + 1 < nbb; s++) {
    if (!master) push(T_LT, s + 1, s, s + 1);
    // the master's step s+1 waits for UPD(s+2, s+2, s) before the step that
    // releases L_{s+1,s+1}, which the TRSMs of column s+1 wait for: listing
    // it first keeps the list topological whatever number of CTAs is resident
    if (master && !clus && s + 2 < nbb) push(T_UPD, s + 2, s + 2, s);
    for (int r = s + 3; r < nbb; r++)
      if (!clus || r != s + 3) push(T_TRSM, r, s + 1, s + 1);
    for (int c = s + 2; c < nbb; c++)
      for (int r = c; r < nbb; r++)
        if (!master || r != s + 2 || c != s + 2) push(T_UPD, r, c, s);  // cluster form: the first helper applies it
  }
}

// ------------------------------------------------------------ panel TRSM
// L_ik = A_ik L_kk^{-T} in FP64 for the listed tiles i > k.  GB300 runs FP64
// at ~2 FMA per clock per SM, so a tile's nb^3 flops are spread over many
// small CTAs: one CTA per (4-row block, tile), 4 warps, warp w = row w, lane =
// column of the current 32-column block cb.  For each cb the solved columns
// are subtracted (L_kk rows staged in shared memory, four independent partial
// sums against the 64-cycle FMA latency), then each warp solves its row
// against the 32x32 diagonal block by forward substitution with shuffles.
constexpr int T64_ROWS = 4;
constexpr int T64_STRIP = 128;
// Optional pre-scaled diagonal blocks (k_trsm64_prep): Ls[(cb*32 + p)*32 + l]
// = L(cb*32 + l, cb*32 + p) / L(cb*32 + p, cb*32 + p) for p < l and rinvs[c] =
// 1 / L(c, c); the block solve then takes one FMA per step (a_l -= a_p Ls)
// and one multiply at the end, where it otherwise scales each x_p first.
// blockIdx.y = z: tile tiles[z] of t64 (or t64 itself when tiles is null),
// outputs in slot z (Ls + z nb 32, rinvs + z nb).
__global__ void k_trsm64_prep(const double *__restrict__ t64, const long *__restrict__ tiles, int nb,
                              double *__restrict__ Ls, double *__restrict__ rinvs, const int *st) {
  if (failed(st)) return;
  __shared__ double rj[B];
  const int cb = blockIdx.x, l = threadIdx.x & (B - 1), p = threadIdx.x >> 5;  // 32 x 32
  const int z = blockIdx.y;
  const double *L = t64 + (tiles ? (size_t)tiles[z] * nb * nb : 0);
  Ls += (size_t)z * nb * B;
  rinvs += (size_t)z * nb;
  const double v = L[(size_t)(cb * B + l) + (size_t)(cb * B + p) * nb];
  if (l == p) {
    const double r = 1.0 / v;
    rj[p] = r;
    rinvs[cb * B + p] = r;
  }
  __syncthreads();
  Ls[(size_t)(cb * B + p) * B + l] = (p < l) ? v * rj[p] : 0.0;
}

// JOBS = false: the tiles (rows[y], k) of one matrix; JOBS = true: explicit
// jobs (batched factor), each with the slot of its pre-scaled L_kk blocks.
// Two instances, so that the single-matrix code does not carry the job path.
template <bool JOBS>
__global__ void __launch_bounds__(128)
    k_trsm64_panel(double *__restrict__ t64, int nb, int NT, int k, const int *__restrict__ rows,
                   const int *st, const int2 *__restrict__ jobs, const double *__restrict__ Ls,
                   const double *__restrict__ rinvs, const int *__restrict__ jslots) {
  if (failed(st)) return;
  extern __shared__ double sm64[];
  const int ldx = nb + 1;
  const int lds = T64_STRIP + 1;
  double *X = sm64;                  // [4][ldx]
  double *S = X + T64_ROWS * ldx;    // [32][lds]
  int r0 = blockIdx.x * T64_ROWS;
  // tiles (i, k) and (k, k) of one matrix, or (batched) explicit tile indices
  long tik, tkk;
  if (JOBS) {
    int2 jb = jobs[blockIdx.y];
    tik = jb.x;
    tkk = jb.y;
    if (Ls) {  // pre-scaled blocks of this job's L_kk
      Ls += (size_t)jslots[blockIdx.y] * nb * B;
      rinvs += (size_t)jslots[blockIdx.y] * nb;
    }
  } else {
    int i = rows ? rows[blockIdx.y] : k + 1 + blockIdx.y;
    tik = tile_index(i, k, NT);
    tkk = tile_index(k, k, NT);
  }
  const double *Lkk = t64 + (size_t)tkk * nb * nb;
  double *A = t64 + (size_t)tik * nb * nb + r0;
  int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll 8
  for (int e = tid; e < T64_ROWS * nb; e += 128) {
    int r = e % T64_ROWS, c = e / T64_ROWS;
    X[r * ldx + c] = A[r + (size_t)c * nb];
  }
  int nbb = nb / B;
  for (int cb = 0; cb < nbb; cb++) {
    const double *Lrow = Lkk + cb * B + lane;  // row cb*32 + lane of L_kk
    double ld[B];
    if (Ls) {
#pragma unroll
      for (int p = 0; p < B; p++) ld[p] = (p < lane) ? Ls[(size_t)(cb * B + p) * B + lane] : 0.0;
    } else {
#pragma unroll
      for (int p = 0; p < B; p++) ld[p] = (p <= lane) ? Lrow[(size_t)(cb * B + p) * nb] : 0.0;
    }
    __syncthreads();
    double a0 = X[w * ldx + cb * B + lane], a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int p0 = 0; p0 < cb * B; p0 += T64_STRIP) {
      int pw = min(T64_STRIP, cb * B - p0);
      {
        double v[T64_STRIP / 4];
#pragma unroll
        for (int u = 0; u < T64_STRIP / 4; u++) {
          int pp = w + 4 * u;
          v[u] = (pp < pw) ? Lrow[(size_t)(p0 + pp) * nb] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < T64_STRIP / 4; u++) {
          int pp = w + 4 * u;
          if (pp < pw) S[lane * lds + pp] = v[u];
        }
      }
      __syncthreads();
      const double *xr = X + w * ldx + p0, *sl = S + lane * lds;
      for (int p = 0; p < pw; p += 4) {
        a0 -= xr[p] * sl[p];
        a1 -= xr[p + 1] * sl[p + 1];
        a2 -= xr[p + 2] * sl[p + 2];
        a3 -= xr[p + 3] * sl[p + 3];
      }
      __syncthreads();
    }
    double a = (a0 + a1) + (a2 + a3);
    if (Ls) {
#pragma unroll
      for (int j = 0; j < B; j++) {
        const double aj = __shfl_sync(0xffffffffu, a, j);
        if (lane > j) a = fma(-aj, ld[j], a);
      }
      a *= rinvs[cb * B + lane];
    } else {
      double mydiag = ld[0];
#pragma unroll
      for (int p = 1; p < B; p++)
        if (p == lane) mydiag = ld[p];
      double myrinv = 1.0 / mydiag;  // off the dependency chain
#pragma unroll
      for (int j = 0; j < B; j++) {
        double rj = __shfl_sync(0xffffffffu, myrinv, j);
        double xj = __shfl_sync(0xffffffffu, a, j) * rj;
        if (lane == j) a = xj;
        if (lane > j) a -= xj * ld[j];
      }
    }
    X[w * ldx + cb * B + lane] = a;
  }
  __syncthreads();
#pragma unroll 8
  for (int e = tid; e < T64_ROWS * nb; e += 128) {
    int r = e % T64_ROWS, c = e / T64_ROWS;
    A[r + (size_t)c * nb] = X[r * ldx + c];
  }
}

// ------------------------------------------------------- trailing update
// C_ij -= L_ik L_jk^T for k < j <= i (SYRK when i == j: lower 64-blocks
// only).  One CTA per (tile pair, 64x64 block), 4x4 outputs per thread,
// K in slices of 16 through shared memory.
constexpr int GM = 64, GK = 16;

__device__ inline void trailing_pair(long q, int m, int *a, int *b) {
  // q-th lower pair (a >= b) of an m x m triangle, packed by column.
  int bb = 0;
  long base = 0;
  while (base + (m - bb) <= q) {
    base += m - bb;
    bb++;
  }
  *b = bb;
  *a = bb + (int)(q - base);
}

__global__ void __launch_bounds__(256)
    k_update64(double *__restrict__ t64, int nb, int NT, int k, const int *st) {
  if (failed(st)) return;
  int m = NT - k - 1;
  int a, b;
  trailing_pair(blockIdx.x, m, &a, &b);
  int i = k + 1 + a, j = k + 1 + b;
  int nsub = nb / GM;
  int bi = blockIdx.y % nsub, bj = blockIdx.y / nsub;
  if (i == j && bi < bj) return;
  const double *Ai = t64 + (size_t)tile_index(i, k, NT) * nb * nb + bi * GM;
  const double *Aj = t64 + (size_t)tile_index(j, k, NT) * nb * nb + bj * GM;
  double *C = t64 + (size_t)tile_index(i, j, NT) * nb * nb + bi * GM + (size_t)bj * GM * nb;
  __shared__ double as[GK][GM];
  __shared__ double bs[GK][GM];
  int t = threadIdx.x, tx = t % 16, ty = t / 16;
  int lc = t / 16, lr = (t % 16) * 4;  // loader: column lc of the slice, rows lr..lr+3
  double acc[4][4] = {};
  for (int p0 = 0; p0 < nb; p0 += GK) {
#pragma unroll
    for (int e = 0; e < 4; e++) {
      as[lc][lr + e] = Ai[(lr + e) + (size_t)(p0 + lc) * nb];
      bs[lc][lr + e] = Aj[(lr + e) + (size_t)(p0 + lc) * nb];
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < GK; p++) {
      double av[4], bv[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        av[e] = as[p][ty + 16 * e];
        bv[e] = bs[p][tx + 16 * e];
      }
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = 0; y < 4; y++) C[(ty + 16 * x) + (size_t)(tx + 16 * y) * nb] -= acc[x][y];
}

// Zero the strict upper triangle of every diagonal tile (they held the
// mirrored covariance), so factor tiles are exactly lower triangular.
__global__ void k_tril_diag(double *__restrict__ t64, int nb, int NT) {
  int k = blockIdx.y;
  double *D = t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  int c = blockIdx.x;
  for (int r = threadIdx.x; r < c; r += blockDim.x) D[r + (size_t)c * nb] = 0.0;
}

// ---------------------------------------------------------------- TRMM
// Y[rows of tile i, samples] = sum_{k <= i} L_ik Z_k in a fixed k order.
// One CTA per (64 rows, 64 samples).
__global__ void __launch_bounds__(256)
    k_trmm64(const double *__restrict__ t64, int n, int nb, int NT,
             const double *__restrict__ Z, long ldz, int s, double *__restrict__ Y,
             long ldy, const unsigned char *__restrict__ cls) {
  int nsub = nb / GM;
  int i = blockIdx.x / nsub, bi = blockIdx.x % nsub;
  int c0 = blockIdx.y * GM;
  __shared__ double as[GK][GM];
  __shared__ double bs[GK][GM];
  int t = threadIdx.x, tx = t % 16, ty = t / 16;
  int lc = t / 16, lr = (t % 16) * 4;    // A loader
  int zc = t / 4, zp = (t % 4) * 4;      // Z loader: sample zc, rows zp..zp+3
  double acc[4][4] = {};
  for (int k = 0; k <= i; k++) {
    if (cls && cls[tile_index(i, k, NT)] != EMU_CLASS_FP64) continue;
    const double *Ai = t64 + (size_t)tile_index(i, k, NT) * nb * nb + bi * GM;
    for (int p0 = 0; p0 < nb; p0 += GK) {
#pragma unroll
      for (int e = 0; e < 4; e++) {
        as[lc][lr + e] = Ai[(lr + e) + (size_t)(p0 + lc) * nb];
        int col = c0 + zc;
        bs[zp + e][zc] = (col < s) ? Z[(size_t)k * nb + p0 + zp + e + (size_t)col * ldz] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < GK; p++) {
        double av[4], bv[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          av[e] = as[p][ty + 16 * e];
          bv[e] = bs[p][tx + 16 * e];
        }
#pragma unroll
        for (int x = 0; x < 4; x++)
#pragma unroll
          for (int y = 0; y < 4; y++) acc[x][y] += av[x] * bv[y];
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int x = 0; x < 4; x++) {
    long gi = (long)i * nb + bi * GM + ty + 16 * x;
    if (gi >= n) continue;
#pragma unroll
    for (int y = 0; y < 4; y++) {
      int col = c0 + tx + 16 * y;
      if (col < s) Y[gi + (size_t)col * ldy] = acc[x][y];
    }
  }
}

// -------------------------------------------------- triangular solves
// Block-row update of the forward solve: X_k -= sum_{j<k} L_kj X_j, and of
// the backward solve: X_k -= sum_{i>k} L_ik^T X_i.  One thread per (row,
// rhs); the sums run over tiles in a fixed order.
__global__ void k_solve_update(const double *__restrict__ t64, int nb, int NT, int k,
                               int backward, double *__restrict__ X, long ldx, int nrhs) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (r >= nb) return;
  double acc = 0.0;
  if (!backward) {
    for (int j = 0; j < k; j++) {
      const double *T = t64 + (size_t)tile_index(k, j, NT) * nb * nb;
      const double *xj = X + (size_t)j * nb + (size_t)c * ldx;
      for (int p = 0; p < nb; p++) acc += T[r + (size_t)p * nb] * xj[p];
    }
  } else {
    for (int i = k + 1; i < NT; i++) {
      const double *T = t64 + (size_t)tile_index(i, k, NT) * nb * nb;
      const double *xi = X + (size_t)i * nb + (size_t)c * ldx;
      for (int p = 0; p < nb; p++) acc += T[p + (size_t)r * nb] * xi[p];
    }
  }
  X[(size_t)k * nb + r + (size_t)c * ldx] -= acc;
}

// Solve with the diagonal tile: one CTA per right-hand side, one thread per
// row; column-oriented substitution (L x = b) or row-oriented (L^T x = b).
__global__ void k_solve_diag(const double *__restrict__ t64, int nb, int NT, int k,
                             int backward, double *__restrict__ X, long ldx) {
  extern __shared__ double xs[];
  int c = blockIdx.x;
  const double *D = t64 + (size_t)tile_index(k, k, NT) * nb * nb;
  double *x = X + (size_t)k * nb + (size_t)c * ldx;
  for (int r = threadIdx.x; r < nb; r += blockDim.x) xs[r] = x[r];
  __syncthreads();
  if (!backward) {
    for (int p = 0; p < nb; p++) {
      double xp = xs[p] / D[p + (size_t)p * nb];
      __syncthreads();
      if (threadIdx.x == 0) xs[p] = xp;
      for (int r = p + 1 + threadIdx.x; r < nb; r += blockDim.x)
        xs[r] -= D[r + (size_t)p * nb] * xp;
      __syncthreads();
    }
  } else {
    for (int p = nb - 1; p >= 0; p--) {
      // x_p = (y_p - sum_{r>p} L[r,p] x_r) / L[p,p]: reduce over r
      double part = 0.0;
      for (int r = p + 1 + threadIdx.x; r < nb; r += blockDim.x)
        part += D[r + (size_t)p * nb] * xs[r];
      __shared__ double red[32];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) sum += red[w];
        xs[p] = (xs[p] - sum) / D[p + (size_t)p * nb];
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < nb; r += blockDim.x) x[r] = xs[r];
}

}  // namespace

extern "C" emu_status emu_potrf_task_list(int nb, int single_tile, int16_t *h_tasks, size_t max_tasks,
                                          size_t *n_tasks) {
  if (nb <= 0 || nb % PB != 0 || nb > 2048 || !n_tasks || (max_tasks > 0 && !h_tasks)) return EMU_EINVAL;
  std::vector<short4> tasks;
  dag_tasks(nb / PB, tasks, single_tile != 0, single_tile == 2);
  *n_tasks = tasks.size();
  const size_t n = tasks.size() < max_tasks ? tasks.size() : max_tasks;
  for (size_t t = 0; t < n; t++) {
    h_tasks[4 * t + 0] = tasks[t].x;
    h_tasks[4 * t + 1] = tasks[t].y;
    h_tasks[4 * t + 2] = tasks[t].z;
    h_tasks[4 * t + 3] = tasks[t].w;
  }
  return EMU_OK;
}

// Ints of the dataflow POTRF workspace for nbat tiles: the task counter and
// each tile's block states, rounded up to a whole number of doubles.
// counter, state[nbb*nbb] per tile, master SM id + 1, CTAs idle on it, the
// helpers' SM ids + 1, CTAs that left theirs; even, so that the pivot
// reciprocals after it are 8-byte aligned
static size_t dag_ws_ints(int nbb, int nbat) {
  size_t n = 6 + (size_t)nbat * nbb * nbb;
  return (n + 1) & ~(size_t)1;
}

emu_status set_dag_wait_hook(emu_ctx *ctx, long long wait_cycles, int withhold_index) {
  const long long cyc = wait_cycles > 0 ? wait_cycles : kDagWaitCycles;
  const int idx = withhold_index >= 0 ? withhold_index : -1;
  EMU_CUDA_TRY(ctx, cudaDeviceSynchronize());
  EMU_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_dag_wait_cycles, &cyc, sizeof(cyc)));
  EMU_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_dag_withhold, &idx, sizeof(idx)));
  return EMU_OK;
}

emu_status launch_potrf64_tile(emu_ctx *ctx, emu_mat *A, int k) {
  return launch_potrf64_ptr(ctx, A->t64 + (size_t)tile_index(k, k, A->nt) * A->nb * A->nb, A->nb, k);
}

emu_status potrf_dag_prepare(emu_ctx *ctx, int nb) {
  int nbb = nb / PB;
  if (ctx->dag_clus < 0) {
    // can a cluster of three CTAs of this kernel be resident?
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(3);
    cfg.blockDim = dim3(PB * PB);
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 3;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_potrf_dag<false>, &cfg);
    ctx->dag_clus = (e == cudaSuccess && nclusters >= 1) ? 1 : 0;
    if (e != cudaSuccess) cudaGetLastError();
  }
  if (ctx->dag_nbb != nbb) {
    std::vector<short4> tasks;
    dag_tasks(nbb, tasks, true, ctx->dag_clus == 1);
    cudaFree(ctx->dag_tasks);
    cudaFree(ctx->dag_ws);
    ctx->dag_tasks = nullptr;
    ctx->dag_ws = nullptr;
    ctx->dag_nbb = 0;
    EMU_CUDA_TRY(ctx, cudaMalloc(&ctx->dag_tasks, tasks.size() * sizeof(short4)));
    EMU_CUDA_TRY(ctx, cudaMemcpy(ctx->dag_tasks, tasks.data(), tasks.size() * sizeof(short4),
                                 cudaMemcpyHostToDevice));
    // counter, state[nbb*nbb], alignment pad, rinv[nb] doubles
    ctx->dag_ws_bytes = dag_ws_ints(nbb, 1) * sizeof(int) + (size_t)nb * sizeof(double);
    EMU_CUDA_TRY(ctx, cudaMalloc(&ctx->dag_ws, ctx->dag_ws_bytes));
    ctx->dag_ntasks = (int)tasks.size();
    ctx->dag_nbb = nbb;
  }
  return EMU_OK;
}

emu_status launch_potrf64_ptr(emu_ctx *ctx, double *D, int nb, int k) {
  int nbb = nb / PB;
  emu_status ps0 = potrf_dag_prepare(ctx, nb);
  if (ps0 != EMU_OK) return ps0;
  ProfScope ps(ctx, PROF_POTRF, (double)nb * nb * nb / 3.0, 16.0 * nb * nb);
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dag_ws, 0, dag_ws_ints(nbb, 1) * sizeof(int), ctx->stream));
  int grid = ctx->sm_count < ctx->dag_ntasks ? ctx->sm_count : ctx->dag_ntasks;
  unsigned long long *trace = nullptr;
  if (ctx->trace_on) {
    // per tile: one record per task, then one per step of the chain's
    // master and of each of its helpers (cluster form)
    const size_t per_tile = (size_t)(ctx->dag_ntasks + 3 * nbb) * 5;
    size_t need = (size_t)(k + 1) * per_tile;
    if (need > ctx->trace_cap) {
      // grow: keep earlier tiles' records of this factor
      unsigned long long *nt = nullptr;
      size_t cap = need * 2;
      EMU_CUDA_TRY(ctx, cudaMallocAsync((void **)&nt, cap * sizeof(unsigned long long), ctx->stream));
      EMU_CUDA_TRY(ctx, cudaMemsetAsync(nt, 0, cap * sizeof(unsigned long long), ctx->stream));
      if (ctx->trace_buf) {
        EMU_CUDA_TRY(ctx, cudaMemcpyAsync(nt, ctx->trace_buf, ctx->trace_cap * sizeof(unsigned long long),
                                          cudaMemcpyDeviceToDevice, ctx->stream));
        cudaFreeAsync(ctx->trace_buf, ctx->stream);
      }
      ctx->trace_buf = nt;
      ctx->trace_cap = cap;
    }
    trace = ctx->trace_buf + (size_t)k * per_tile;
    ctx->trace_records = (size_t)(k + 1) * (ctx->dag_ntasks + 3 * nbb);
  }
  double *rinv = reinterpret_cast<double *>(ctx->dag_ws + dag_ws_ints(nbb, 1));
  if (ctx->dag_clus == 1) {
    // the chain on cluster 0 (three CTAs), the tasks on the other clusters;
    // two workers per SM: the task throughput paces the chain
    int g = ctx->dag_ntasks + 2 < 2 * ctx->sm_count ? ctx->dag_ntasks + 2 : 2 * ctx->sm_count;
    g = (g + 2) / 3 * 3;
    if (g < 6) g = 6;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(PB * PB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 3;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    EMU_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, k_potrf_dag<false>, D, nb, k * nb, (const short4 *)ctx->dag_tasks,
                                         ctx->dag_ntasks, ctx->dag_ws, rinv, ctx->d_status, trace,
                                         (const long *)nullptr, 1, (int *)nullptr));
  } else {
    k_potrf_dag<false><<<grid, PB * PB, 0, ctx->stream>>>(D, nb, k * nb, (const short4 *)ctx->dag_tasks,
                                                         ctx->dag_ntasks, ctx->dag_ws, rinv, ctx->d_status, trace,
                                                         nullptr, 1, nullptr);
  }
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trsm64_jobs(emu_ctx *ctx, double *t64, int nb, const int2 *d_jobs, int njobs, const double *Ls,
                              const double *rinvs, const int *d_jslots) {
  if (njobs <= 0) return EMU_OK;
  double nb3 = (double)nb * nb * nb;
  ProfScope ps(ctx, PROF_TRSM64, njobs * nb3, 16.0 * njobs * nb * nb);
  size_t sm = (size_t)(T64_ROWS * (nb + 1) + 32 * (T64_STRIP + 1)) * sizeof(double);
  EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsm64_panel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_trsm64_panel<true><<<dim3(nb / T64_ROWS, njobs), 128, sm, ctx->stream>>>(t64, nb, 0, 0, nullptr, ctx->d_status,
                                                                            d_jobs, Ls, rinvs, d_jslots);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

size_t potrf_dag_task_count(int nb) {
  std::vector<short4> tasks;
  dag_tasks(nb / PB, tasks, false);
  return tasks.size();
}

emu_status potrf_dag_tasks_upload(emu_ctx *ctx, int nb, void *d_tasks, cudaStream_t s) {
  std::vector<short4> tasks;
  dag_tasks(nb / PB, tasks, false);
  EMU_CUDA_TRY(ctx, cudaMemcpyAsync(d_tasks, tasks.data(), tasks.size() * sizeof(short4), cudaMemcpyHostToDevice, s));
  // the host vector goes out of scope: wait for the copy
  EMU_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return EMU_OK;
}

size_t potrf_batch_ws_ints(int nb, int nbat) { return dag_ws_ints(nb / PB, nbat); }

emu_status launch_potrf64_batch(emu_ctx *ctx, double *t64, int nb, int k, const long *d_tiles, int nbat,
                                const void *d_tasks, int ntasks, int *ws, double *rinv, int *bad) {
  if (nbat <= 0) return EMU_OK;
  int nbb = nb / PB;
  ProfScope ps(ctx, PROF_POTRF, (double)nbat * nb * nb * nb / 3.0, 16.0 * nbat * nb * nb);
  EMU_CUDA_TRY(ctx, cudaMemsetAsync(ws, 0, dag_ws_ints(nbb, nbat) * sizeof(int), ctx->stream));
  long total = (long)ntasks * nbat;
  int grid = (int)std::min<long>(total, 4L * ctx->sm_count);
  k_potrf_dag<true><<<grid, PB * PB, 0, ctx->stream>>>(t64, nb, k * nb, (const short4 *)d_tasks, ntasks, ws,
                                                      rinv, ctx->d_status, nullptr, d_tiles, nbat, bad);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trsm64_prep(emu_ctx *ctx, const double *L, int nb, double *Ls, double *rinvs, const long *d_tiles,
                              int n) {
  if (nb % B != 0) return EMU_EINVAL;
  if (n <= 0) return EMU_OK;
  ProfScope ps(ctx, PROF_SPLIT, 0.0, 16.0 * n * (double)nb * B);
  k_trsm64_prep<<<dim3(nb / B, n), B * B, 0, ctx->stream>>>(L, d_tiles, nb, Ls, rinvs, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trsm64_panel(emu_ctx *ctx, emu_mat *A, int k, const int *d_rows, int nrows, const double *Ls,
                               const double *rinvs) {
  int m = d_rows ? nrows : A->nt - k - 1;
  if (m <= 0) return EMU_OK;
  double nb3 = (double)A->nb * A->nb * A->nb;
  ProfScope ps(ctx, PROF_TRSM64, m * nb3, 16.0 * m * A->nb * A->nb);
  size_t sm = (size_t)(T64_ROWS * (A->nb + 1) + 32 * (T64_STRIP + 1)) * sizeof(double);
  EMU_CUDA_TRY(ctx, cudaFuncSetAttribute(k_trsm64_panel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_trsm64_panel<false><<<dim3(A->nb / T64_ROWS, m), 128, sm, ctx->stream>>>(A->t64, A->nb, A->nt, k, d_rows,
                                                                            ctx->d_status, nullptr, Ls, rinvs, nullptr);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_update64(emu_ctx *ctx, emu_mat *A, int k) {
  int m = A->nt - k - 1;
  if (m <= 0) return EMU_OK;
  long pairs = (long)m * (m + 1) / 2;
  int nsub = A->nb / GM;
  double nb3 = (double)A->nb * A->nb * A->nb;
  ProfScope ps(ctx, PROF_UPDATE64, (double)m * m * nb3, 8.0 * A->nb * A->nb * (2.0 * pairs + 2.0 * m));
  k_update64<<<dim3((unsigned)pairs, nsub * nsub), 256, 0, ctx->stream>>>(
      A->t64, A->nb, A->nt, k, ctx->d_status);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_tril_diag(emu_ctx *ctx, emu_mat *A) {
  k_tril_diag<<<dim3(A->nb, A->nt), 128, 0, ctx->stream>>>(A->t64, A->nb, A->nt);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

emu_status launch_trmm64(emu_ctx *ctx, const emu_mat *L, const double *Z, long ldz,
                         int s, double *Y, long ldy, const unsigned char *cls) {
  dim3 grid(L->nt * (L->nb / GM), (s + GM - 1) / GM);
  ProfScope ps(ctx, PROF_TRMM64, (double)L->n * L->n * s, 8.0 * tile_count(L->nt) * L->nb * L->nb);
  k_trmm64<<<grid, 256, 0, ctx->stream>>>(L->t64, L->n, L->nb, L->nt, Z, ldz, s, Y, ldy, cls);
  EMU_LAUNCHED(ctx);
  return EMU_OK;
}

// X (npad x nrhs, ld ldx >= npad, padded rows zero) <- (L L^T)^{-1} X.
emu_status launch_potrs64(emu_ctx *ctx, const emu_mat *L, double *X, long ldx, int nrhs) {
  int nb = L->nb, NT = L->nt;
  int thr = 256;
  ProfScope ps(ctx, PROF_SOLVE, 2.0 * L->n * L->n * nrhs, 16.0 * tile_count(NT) * nb * nb);
  for (int k = 0; k < NT; k++) {
    if (k > 0) {
      k_solve_update<<<dim3((nb + thr - 1) / thr, nrhs), thr, 0, ctx->stream>>>(
          L->t64, nb, NT, k, 0, X, ldx, nrhs);
      EMU_LAUNCHED(ctx);
    }
    k_solve_diag<<<nrhs, 512, nb * sizeof(double), ctx->stream>>>(L->t64, nb, NT, k, 0, X, ldx);
    EMU_LAUNCHED(ctx);
  }
  for (int k = NT - 1; k >= 0; k--) {
    if (k < NT - 1) {
      k_solve_update<<<dim3((nb + thr - 1) / thr, nrhs), thr, 0, ctx->stream>>>(
          L->t64, nb, NT, k, 1, X, ldx, nrhs);
      EMU_LAUNCHED(ctx);
    }
    k_solve_diag<<<nrhs, 512, nb * sizeof(double), ctx->stream>>>(L->t64, nb, NT, k, 1, X, ldx);
    EMU_LAUNCHED(ctx);
  }
  return EMU_OK;
}
