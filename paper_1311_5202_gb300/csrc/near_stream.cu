// Near-field apply (the direct and corrected near sum of Eq. kcorrection) as a bulk-copy stream.
//
// Every target leaf's direct blocks form one contiguous column-major matrix (rows: the leaf's points,
// columns: the points of its direct source boxes), 4-entry aligned in HBM. A persistent grid of CTAs
// (three per SM) owns balanced, contiguous ranges of target leaves. In each CTA one producer thread walks
// the leaves' matrices chunk by chunk (whole columns, <= 16 KB) and issues cp.async.bulk copies into a
// ring of shared-memory stages (three, or four for batches), each guarded by a "full" mbarrier (transaction
// bytes) and an "empty" mbarrier (one arrival per consumer warp). Eight consumer warps bring the leaf's source
// densities into shared memory per column window (one index per column), then read each landed stage: thread
// (i, g) takes row i and columns g, g + G, ... (G = 256 / rows), so consecutive threads read consecutive
// shared-memory words. Group partial sums are reduced per row.
//
// The correction entries that fall outside the leaf's direct blocks (a CSR per row, one contiguous range per
// leaf) are applied in one of three schedules, chosen per plan by timing:
//  0: inside the stream: spread over all consumer threads, summed per row by a segmented warp scan;
//  1: by k_near_corr before the stream (one warp per row); the stream adds its sums to y;
//  2: as 1, with the density windows double-buffered: the next window's densities are copied with cp.async
//     while the current one is used, and its column indices are loaded a window ahead.
// 16 right-hand sides per pass always run as 2.
//
// Every wait is bounded: a wait that gives up sets the error flag, the kernel runs to its end without
// touching other memory, and the producer still waits (bounded) for its own copies in flight.
#include "plan.cuh"

namespace fda {

#define NS_STAGE_BYTES 16384
#define NS_CONS 256            // consumer threads (8 warps)
#define NS_NT (NS_CONS + 32)   // + one producer warp
#define NS_WAIT_NS 1000000000ull  // 1 s

__device__ __forceinline__ uint32_t ns_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// wait on the mbarrier phase with a wall-clock bound of 1 s; returns false when it gives up
__device__ __forceinline__ bool ns_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = ns_smem(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    uint64_t now;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(now));
    if (it == 0) t0 = now;
    else if (now - t0 > NS_WAIT_NS) return false;
  }
}

__device__ __forceinline__ void ns_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(ns_smem(bar)) : "memory");
}

__device__ __forceinline__ void ns_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(ns_smem(bar)),
               "r"(bytes)
               : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completion on an mbarrier
__device__ __forceinline__ void ns_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   ns_smem(dst)),
               "l"(src), "r"(bytes), "r"(ns_smem(bar))
               : "memory");
}

// the same copy with an L2 policy (the near-field matrices are read once per pass: evict them first, so that
// they do not push out what other kernels of the product keep in L2)
__device__ __forceinline__ void ns_bulk_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                             uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(ns_smem(dst)),
      "l"(src), "r"(bytes), "r"(ns_smem(bar)), "l"(pol)
      : "memory");
}

// global -> shared asynchronous copies of densities (zero-filled beyond src_bytes)
__device__ __forceinline__ void ns_cp8(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(ns_smem(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void ns_cp16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(ns_smem(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

// barrier among the consumer warps only (the producer warp never joins it)
__device__ __forceinline__ void ns_cons_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NS_CONS) : "memory"); }

// single right-hand side: three CTAs per SM (3-stage ring, 16 KB density window); batches: fewer, larger CTAs
// Double-buffered density windows (DB): two windows, the next one copied with cp.async while the current one
// is used; corrections always by the separate CSR kernel (no correction buffer). 16 right-hand sides per pass
// always run this way (two windows of at most 256 columns, 32 KB each); one right-hand side does when W is set
// (two windows of 8 KB: 1024 FP32 or 512 FP64 columns, several per thread).
// D (FP32, one right-hand side only): a deeper ring of four stages that still fits three CTAs per SM (each CTA
// at 76,768 bytes of the 76,800 that three CTAs may take); the stage shrinks to 14,272 or 13,760 bytes. FP64
// products keep the three-stage ring.
// D = 2 (FP32, one right-hand side, double-buffered windows): each density is kept in the window as
// (x.x, x.x, x.y, x.y), so that a complex entry b costs two packed FP32x2 FMAs, b (x.x, x.x) and b (x.y, x.y),
// into two accumulators that give the complex sum at the leaf's end; 512 columns per window.
template <typename C, int NR, bool W = false, int D = 0>
struct NsLayout {
  static constexpr int E = sizeof(C);
  static constexpr bool DB = NR == 16 || W;
  static constexpr bool DEEP = D == 1 && NR == 1 && E == 8;
  static constexpr bool X2 = D == 2 && NR == 1 && E == 8 && W;
  // D = 2 with several right-hand sides (FP32): the matrix entry b is paired in registers, (b.x, b.x) and
  // (b.y, b.y), and each density x of the pass takes two packed FMAs into two accumulators
  static constexpr bool PK = D == 2 && NR > 1 && E == 8;
  // D = 3 (FP32, one right-hand side, double-buffered windows): a slim CTA of about 47 KB (three 12 KB stages,
  // two 4 KB windows) for products whose far field runs beside the near field and needs the shared memory
  static constexpr bool SLIM = D == 3 && NR == 1 && E == 8 && W;
  static constexpr int XE = X2 ? 16 : NR * E;  // window bytes per column
  static constexpr int SB = DEEP ? (W ? 14272 : 13760) : (SLIM ? 12288 : NS_STAGE_BYTES);  // multiple of 16
  static constexpr int STAGES = NR == 1 ? (DEEP ? 4 : 3) : 4;
  static constexpr int MINB = NR == 1 ? 3 : (NR <= 4 ? 2 : 1);
  static constexpr int XBYTES =
      NR == 16 ? 32768 : (W ? (SLIM ? 4096 : 8192) : ((NR == 1 || E * NR >= 64) ? 16384 : 32768));
  static constexpr int XW0 = (XBYTES / XE) & ~1;
  static constexpr int XW = NR == 16 && XW0 > NS_CONS ? NS_CONS : XW0;  // columns per density window (even)
  static constexpr int CPT = DB && XW > NS_CONS ? XW / NS_CONS : 1;     // window columns per consumer thread
  static_assert(!DB || XW <= NS_CONS || XW % NS_CONS == 0, "double-buffered window: whole columns per thread");
  static constexpr size_t ring = (size_t)STAGES * SB;
  static constexpr size_t xs = ring;
  static constexpr size_t red = xs + (size_t)(DB ? 2 : 1) * XW * XE;
  static constexpr size_t cor = red + (size_t)NS_CONS * NR * E;
  static constexpr size_t crow = cor + (DB ? (size_t)0 : (size_t)NS_CONS * NR * E);
  static constexpr size_t bars = crow + (NS_CONS + 8) * sizeof(int);
  static constexpr size_t total = bars + 2 * STAGES * sizeof(uint64_t) + 128;  // + alignment slack
  static_assert(!DEEP || total <= 76800, "the deep ring must leave room for three CTAs per SM");
};

// columns per chunk: whole columns, an even count, at most one stage
__device__ __forceinline__ int ns_cpc(int nr, int E, int sb) { return max(2, (sb / (nr * E)) & ~1); }

template <typename C, int NR, bool W, int D>
static __global__ void __launch_bounds__(NS_NT, NsLayout<C, NR, W, D>::MINB) k_near_stream(
    const int32_t* part, const NsMeta* meta, const int32_t* ncolv, const int64_t* xbase, const int32_t* xcol,
    const C* B, const int64_t* cptr, const int32_t* ccol, const C* cval, const C* xt, const float4* xdup, C* yt,
    int nrhs, int r0, int rc, int csep, int evict_first, int* err) {
  typedef NsLayout<C, NR, W, D> Ly;
  typedef decltype(xt[0].x) R;
  constexpr int E = Ly::E, XW = Ly::XW, NS_STAGES = Ly::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)((((uintptr_t)smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char* ring = sm;
  C* xs = (C*)(sm + Ly::xs);
  C* red = (C*)(sm + Ly::red);
  C* cor = (C*)(sm + Ly::cor);
  int* crow = (int*)(sm + Ly::crow);
  uint64_t* full = (uint64_t*)(sm + Ly::bars);
  uint64_t* empty = full + NS_STAGES;
  const int t = threadIdx.x;
  if (t == 0) {
    for (int s = 0; s < NS_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ns_smem(&full[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ns_smem(&empty[s])), "r"(NS_CONS / 32));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const int u0 = part[blockIdx.x], u1 = part[blockIdx.x + 1];

  if (t >= NS_CONS) {
    // ---------------- producer
    if (t == NS_CONS) {
      int it = 0;
      bool ok = true;
      uint64_t pol = 0;
      if (evict_first) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
      NsMeta mn;  // the next leaf's description, loaded while this leaf's copies are issued
      if (u0 < u1) mn = meta[u0];
      for (int u = u0; u < u1 && ok; ++u) {
        const NsMeta m = mn;
        if (u + 1 < u1) mn = meta[u + 1];
        const int nr = m.nr;
        const int ncol = m.ncol;
        const unsigned char* src = (const unsigned char*)(B + m.nb);
        const int cpc = ns_cpc(nr, E, Ly::SB);
        for (int c = 0; c < ncol;) {
          const int wend = min(ncol, (c / XW + 1) * XW);
          const int cc = min(cpc, wend - c);
          const int st = it % NS_STAGES;
          if (it >= NS_STAGES && !ns_wait(&empty[st], ((it / NS_STAGES) - 1) & 1)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          const uint32_t bytes = (uint32_t)(((int64_t)cc * nr * E + 15) & ~(int64_t)15);
          ns_expect_tx(&full[st], bytes);
          if (evict_first)
            ns_bulk_hint(ring + (size_t)st * Ly::SB, src + (int64_t)c * nr * E, bytes, &full[st], pol);
          else
            ns_bulk(ring + (size_t)st * Ly::SB, src + (int64_t)c * nr * E, bytes, &full[st]);
          c += cc;
          ++it;
        }
      }
      // the last fill of every stage has landed before the CTA's shared memory is released
      for (int j = max(0, it - NS_STAGES); j < it; ++j) ns_wait(&full[j % NS_STAGES], (j / NS_STAGES) & 1);
    }
    return;
  }

  // ---------------- consumers
  const int lane = t & 31;
  int it = 0;
  bool failed = false;
  // double-buffered windows: window A is the next one to copy; colA[] are this thread's columns of it (column
  // t + j * 256), loaded one window ahead so that their latency hides behind the current window's work
  constexpr int CPT = Ly::CPT;
  int ua = u0, wa = 0, buf = 0;
  int colA[CPT];
  auto load_cols = [&]() {
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int k = t + j * NS_CONS, c = wa + k;
      colA[j] = (ua < u1 && k < XW && c < ncolv[ua]) ? xcol[xbase[ua] + c] : -1;
    }
  };
  // next window in the consumers' order (leaves without columns have no window)
  auto normalize = [&]() {
    while (ua < u1 && wa >= ncolv[ua]) {
      ++ua;
      wa = 0;
    }
  };
  auto advance = [&]() {
    wa += XW;
    normalize();
  };
  auto copy_window = [&](int b) {
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int col = colA[j];
      if (col < 0) continue;
      if constexpr (Ly::X2) {  // the duplicated densities, 16 bytes a column
        ns_cp16((float4*)xs + ((size_t)b * XW + t + j * NS_CONS), xdup + col, 16u);
        continue;
      }
      C* dst = xs + ((size_t)b * XW + t + j * NS_CONS) * NR;
      const C* src = xt + (int64_t)col * nrhs + r0;
      if (E == 16 || (NR > 1 && (nrhs & 1) == 0)) {  // 16-byte aligned runs of 16 / E right-hand sides
        constexpr int V = E == 16 ? 1 : 2;
#pragma unroll
        for (int q = 0; q < NR; q += V) {
          const int nb = min(16, max(0, (rc - q) * E));
          ns_cp16(dst + q, nb > 0 ? (const void*)(src + q) : (const void*)xt, (uint32_t)nb);
        }
      } else {
#pragma unroll
        for (int q = 0; q < NR; ++q) ns_cp8(dst + q, q < rc ? (const void*)(src + q) : (const void*)xt, q < rc ? 8u : 0u);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if constexpr (Ly::DB) {
    normalize();
    load_cols();
    copy_window(0);  // window 0
    advance();
    load_cols();
  }
  // FP32: each leaf's description is loaded one leaf ahead, so that no leaf starts on a global load (FP64 has
  // no registers to spare for it)
  NsMeta mnext;
  if (E == 8 && u0 < u1) mnext = meta[u0];
  for (int u = u0; u < u1; ++u) {
    NsMeta m;
    if constexpr (E == 8) {
      m = mnext;
      if (u + 1 < u1) mnext = meta[u + 1];
    } else {
      m = meta[u];
    }
    const int64_t tb = m.tb;
    const int nr = m.nr;
    const int ncol = m.ncol;
    const int64_t xb = m.xb;
    const int cpc = ns_cpc(nr, E, Ly::SB);
    // split schedule: the correction sums that k_near_corr stored for this leaf's rows, read now and added at
    // the leaf's end
    const bool ypre_ok = E == 8 && csep && nr * rc <= NS_CONS;  // FP64: registers are short
    C ypre = mk((R)0, (R)0);
    if (ypre_ok && t < nr * rc) {
      const int r = t / rc, rr = t - r * rc;
      ypre = yt[(tb + r) * nrhs + r0 + rr];
    }
    const int G = NS_CONS / nr;
    const int i = t % nr, g = t / nr;
    const bool act = g < G;
    // correction entries outside the direct blocks. A leaf's rows are consecutive, so its entries are one
    // CSR range: every thread takes entries, finds the row by binary search over the leaf's row pointers
    // and adds into shared memory (one parallel pass instead of a chain per row).
    const int64_t cb = csep ? 0 : cptr[tb];
    if (!csep) {
      for (int q = t; q <= nr; q += NS_CONS) crow[q] = (int)(cptr[tb + q] - cb);
      for (int q = t; q < nr * NR; q += NS_CONS) cor[q] = mk((R)0, (R)0);
      ns_cons_sync();
    }
    const int ncor = csep ? 0 : crow[nr];
    constexpr int CE = NR <= 4 ? 4 : 1;  // correction entries per thread and pass (register budget)
    for (int e0 = 0; e0 < ncor; e0 += CE * NS_CONS) {
      // all loads first (CE entries per thread), then the density gathers, then per-entry products
      C v[CE];
      int col[CE];
#pragma unroll
      for (int j = 0; j < CE; ++j) {
        const int e = e0 + j * NS_CONS + t;
        v[j] = e < ncor ? cval[cb + e] : mk((R)0, (R)0);
        col[j] = e < ncor ? ccol[cb + e] : 0;
      }
      C xv[CE][NR];
#pragma unroll
      for (int j = 0; j < CE; ++j)
#pragma unroll
        for (int q = 0; q < NR; ++q)
          xv[j][q] = (e0 + j * NS_CONS + t < ncor && q < rc) ? xt[(int64_t)col[j] * nrhs + r0 + q] : mk((R)0, (R)0);
#pragma unroll
      for (int j = 0; j < CE; ++j) {
        const int e = e0 + j * NS_CONS + t;
        int row = -1;  // largest r with crow[r] <= e (rows are non-decreasing along the lanes)
        if (e < ncor) {
          int lo = 0, hi = nr;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (crow[mid] <= e) lo = mid; else hi = mid;
          }
          row = lo;
        }
        C a[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          a[q] = mk((R)0, (R)0);
          cfma(a[q], v[j], xv[j][q]);
        }
        // segmented inclusive scan over lanes of equal row; the last lane of each segment holds its sum
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int ro = __shfl_up_sync(0xffffffffu, row, off);
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const R ax = __shfl_up_sync(0xffffffffu, a[q].x, off);
            const R ay = __shfl_up_sync(0xffffffffu, a[q].y, off);
            if (lane >= off && ro == row) {
              a[q].x += ax;
              a[q].y += ay;
            }
          }
        }
        const int rn = __shfl_down_sync(0xffffffffu, row, 1);
        if (row >= 0 && (lane == 31 || rn != row)) {
#pragma unroll
          for (int q = 0; q < NR; ++q)
            if (q < rc) {
              atomicAdd(&cor[row * NR + q].x, a[q].x);
              atomicAdd(&cor[row * NR + q].y, a[q].y);
            }
        }
      }
    }
    C acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = mk((R)0, (R)0);
    float2 accA = make_float2(0.f, 0.f), accB = make_float2(0.f, 0.f);  // X2: sums of b x.x and b x.y
    float2 pkP[Ly::PK ? NR : 1], pkQ[Ly::PK ? NR : 1];  // PK: sums of b.x x and b.y x per right-hand side
#pragma unroll
    for (int q = 0; q < (Ly::PK ? NR : 1); ++q) pkP[q] = pkQ[q] = make_float2(0.f, 0.f);
    for (int wb = 0; wb < ncol; wb += XW) {
      const int we = min(ncol, wb + XW);
      const C* xcur = xs;
      if constexpr (Ly::DB) {
        // this window's copies have landed (own, then everyone's); the other buffer's readers are done
        asm volatile("cp.async.wait_all;" ::: "memory");
        ns_cons_sync();
        copy_window(buf ^ 1);
        advance();
        load_cols();
        xcur = (const C*)((const unsigned char*)xs + (size_t)buf * XW * Ly::XE);
        buf ^= 1;
      } else {
        ns_cons_sync();  // readers of the previous window are done
        for (int c = wb + t; c < we; c += NS_CONS) {
          const C* xp = xt + (int64_t)xcol[xb + c] * nrhs + r0;
#pragma unroll
          for (int q = 0; q < NR; ++q) xs[(c - wb) * NR + q] = (q < rc) ? xp[q] : mk((R)0, (R)0);
        }
        ns_cons_sync();
      }
      for (int c = wb; c < we;) {
        const int cc = min(cpc, we - c);
        const int st = it % NS_STAGES;
        if (!failed && !ns_wait(&full[st], (it / NS_STAGES) & 1)) {
          failed = true;
          atomicExch(err, 1);
        }
        if constexpr (Ly::X2) {
          if (!failed && act) {
            const float2* Bs = (const float2*)(ring + (size_t)st * Ly::SB) + i;
            const float4* xw = (const float4*)xcur + (c - wb);
            int cl = g;
            for (; cl + 3 * G < cc; cl += 4 * G) {
              const float2 b0 = Bs[cl * nr], b1 = Bs[(cl + G) * nr], b2 = Bs[(cl + 2 * G) * nr],
                           b3 = Bs[(cl + 3 * G) * nr];
              const float4 x0 = xw[cl], x1 = xw[cl + G], x2 = xw[cl + 2 * G], x3 = xw[cl + 3 * G];
              accA = __ffma2_rn(b0, make_float2(x0.x, x0.y), accA);
              accB = __ffma2_rn(b0, make_float2(x0.z, x0.w), accB);
              accA = __ffma2_rn(b1, make_float2(x1.x, x1.y), accA);
              accB = __ffma2_rn(b1, make_float2(x1.z, x1.w), accB);
              accA = __ffma2_rn(b2, make_float2(x2.x, x2.y), accA);
              accB = __ffma2_rn(b2, make_float2(x2.z, x2.w), accB);
              accA = __ffma2_rn(b3, make_float2(x3.x, x3.y), accA);
              accB = __ffma2_rn(b3, make_float2(x3.z, x3.w), accB);
            }
            for (; cl < cc; cl += G) {
              const float2 bv = Bs[cl * nr];
              const float4 xv = xw[cl];
              accA = __ffma2_rn(bv, make_float2(xv.x, xv.y), accA);
              accB = __ffma2_rn(bv, make_float2(xv.z, xv.w), accB);
            }
          }
        } else if constexpr (Ly::PK) {
          if (!failed && act) {
            const float2* Bs = (const float2*)(ring + (size_t)st * Ly::SB) + i;
            const float2* xw = (const float2*)xcur + (c - wb) * NR;
            int cl = g;
            for (; cl + G < cc; cl += 2 * G) {
              const float2 b0 = Bs[cl * nr], b1 = Bs[(cl + G) * nr];
              const float2 bx0 = make_float2(b0.x, b0.x), by0 = make_float2(b0.y, b0.y);
              const float2 bx1 = make_float2(b1.x, b1.x), by1 = make_float2(b1.y, b1.y);
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                const float2 x0 = xw[cl * NR + q], x1 = xw[(cl + G) * NR + q];
                pkP[q] = __ffma2_rn(bx0, x0, pkP[q]);
                pkQ[q] = __ffma2_rn(by0, x0, pkQ[q]);
                pkP[q] = __ffma2_rn(bx1, x1, pkP[q]);
                pkQ[q] = __ffma2_rn(by1, x1, pkQ[q]);
              }
            }
            for (; cl < cc; cl += G) {
              const float2 b0 = Bs[cl * nr];
              const float2 bx0 = make_float2(b0.x, b0.x), by0 = make_float2(b0.y, b0.y);
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                const float2 x0 = xw[cl * NR + q];
                pkP[q] = __ffma2_rn(bx0, x0, pkP[q]);
                pkQ[q] = __ffma2_rn(by0, x0, pkQ[q]);
              }
            }
          }
        } else if (!failed && act) {
          const C* Bs = (const C*)(ring + (size_t)st * Ly::SB) + i;
          const C* xw = xcur + (c - wb) * NR;
          int cl = g;
          for (; cl + 3 * G < cc; cl += 4 * G) {
            const C b0 = Bs[cl * nr], b1 = Bs[(cl + G) * nr], b2 = Bs[(cl + 2 * G) * nr], b3 = Bs[(cl + 3 * G) * nr];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              cfma(acc[q], b0, xw[cl * NR + q]);
              cfma(acc[q], b1, xw[(cl + G) * NR + q]);
              cfma(acc[q], b2, xw[(cl + 2 * G) * NR + q]);
              cfma(acc[q], b3, xw[(cl + 3 * G) * NR + q]);
            }
          }
          for (; cl < cc; cl += G) {
            const C bv = Bs[cl * nr];
#pragma unroll
            for (int q = 0; q < NR; ++q) cfma(acc[q], bv, xw[cl * NR + q]);
          }
        }
        __syncwarp();
        if (lane == 0) ns_arrive(&empty[st]);
        c += cc;
        ++it;
      }
    }
    // X2: b x = (b.x x.x - b.y x.y, b.y x.x + b.x x.y) from the two packed sums
    if constexpr (Ly::X2) acc[0] = mk(accA.x - accB.y, accA.y + accB.x);
    if constexpr (Ly::PK) {  // b x = (b.x x.x - b.y x.y, b.x x.y + b.y x.x)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] = mk(pkP[q].x - pkQ[q].y, pkP[q].y + pkQ[q].x);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) red[t * NR + q] = act ? acc[q] : mk((R)0, (R)0);
    ns_cons_sync();
    for (int q = t; q < nr * rc; q += NS_CONS) {
      const int r = q / rc, rr = q - r * rc;
      C* yp = yt + (tb + r) * nrhs + r0 + rr;
      C s = csep ? (ypre_ok ? ypre : *yp) : cor[r * NR + rr];
      for (int gg = 0; gg < G; ++gg) s = cadd(s, red[(gg * nr + r) * NR + rr]);
      *yp = s;
    }
    ns_cons_sync();  // red and cor are rewritten by the next leaf
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy in flight when the CTA exits
}

// Correction entries outside the direct blocks as their own CSR product (tree order), run before the stream
// when the plan chooses it: one warp per row, lanes over the row's entries, NR right-hand sides per pass. The
// lane sums are reduced by recursive halving (each exchange step keeps half of the right-hand sides on each
// side of the butterfly), so NR = 16 needs 32 shuffles per row instead of 16 full reductions. The row sums
// are stored into y; the stream then adds its direct-block sums to them.
template <typename C, int NR>
static __global__ void __launch_bounds__(256) k_near_corr(const int64_t* cptr, const int32_t* ccol, const C* cval,
                                                          const C* xt, C* yt, int64_t N, int nrhs, int r0, int rc) {
  typedef decltype(xt[0].x) R;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  const int64_t e0 = cptr[row], e1 = cptr[row + 1];
  C a[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) a[q] = mk((R)0, (R)0);
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    const C v = cval[e];
    const C* xp = xt + (int64_t)ccol[e] * nrhs + r0;
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (q < rc) cfma(a[q], v, xp[q]);
  }
  // recursive halving: after the step at lane distance off, a lane keeps the upper or lower half of its
  // right-hand sides (by its lane bit) and adds the partner's copy of that half
  int qi = 0;
  int off = 16;
#pragma unroll
  for (int w = NR; w > 1; w >>= 1, off >>= 1) {
    const int h = w >> 1;
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const C send = hi ? a[i] : a[i + h];
      const C keep = hi ? a[i + h] : a[i];
      a[i] = mk(keep.x + __shfl_xor_sync(0xffffffffu, send.x, off), keep.y + __shfl_xor_sync(0xffffffffu, send.y, off));
    }
    if (hi) qi += h;
  }
  for (; off >= 1; off >>= 1) {
    a[0].x += __shfl_xor_sync(0xffffffffu, a[0].x, off);
    a[0].y += __shfl_xor_sync(0xffffffffu, a[0].y, off);
  }
  // lanes whose remaining (fully reduced) bits are zero hold right-hand side qi
  constexpr int LOGNR = NR == 1 ? 0 : (NR == 4 ? 2 : 4);
  if ((lane & ((1 << (5 - LOGNR)) - 1)) == 0 && qi < rc) yt[row * nrhs + r0 + qi] = a[0];
}

static __global__ void k_dup_x(const float2* xt, float4* xdup, int64_t N) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    const float2 v = xt[i];
    xdup[i] = make_float4(v.x, v.x, v.y, v.y);
  }
}

template <typename C, int NR, bool W, int D = 0>
static int near_stream_t(fda_plan_s* P, const C* B, const C* cval, const C* xt, C* yt, int nrhs, cudaStream_t s,
                         int64_t* launches) {
  typedef NsLayout<C, NR, W, D> Ly;
  static bool attr = false;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_near_stream<C, NR, W, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Ly::total));
    attr = true;
  }
  fda_tree_s* T = P->tree;
  const int csep = (Ly::DB || P->near_csep >= 1) ? 1 : 0;  // double-buffered passes have no correction buffer
  const float4* xdup = nullptr;
  if constexpr (Ly::X2) {  // (x.x, x.x, x.y, x.y) per point for the packed FMAs
    k_dup_x<<<(unsigned)((T->N + 255) / 256), 256, 0, s>>>((const float2*)xt, P->xdup32.p, T->N);
    FDA_LAUNCH_CHECK();
    ++*launches;
    xdup = P->xdup32.p;
  }
  for (int r0 = 0; r0 < nrhs; r0 += NR) {
    const int rc = std::min(NR, nrhs - r0);
    if (csep) {
      k_near_corr<C, NR><<<(unsigned)((T->N + 7) / 8), 256, 0, s>>>(P->corr_ptr.p, P->corr_col.p, cval, xt, yt, T->N,
                                                                    nrhs, r0, rc);
      FDA_LAUNCH_CHECK();
      ++*launches;
    }
    const int ov = (P->near_sel == 1 || P->near_sel == 2) && P->near_grid_ov[P->near_sel - 1] > 0 ? P->near_sel : 0;
    k_near_stream<C, NR, W, D><<<(unsigned)(ov ? P->near_grid_ov[ov - 1] : P->near_grid), NS_NT, Ly::total, s>>>(
        ov ? P->near_part_ov[ov - 1].p : P->near_part.p, P->near_meta.p, P->near_ncol.p, P->near_xbase.p,
        P->near_xcol.p, B, P->corr_ptr.p, P->corr_col.p, cval, xt, xdup, yt, nrhs, r0, rc, csep, P->near_evict,
        P->tc_err.p);
    FDA_LAUNCH_CHECK();
    ++*launches;
  }
  return FDA_OK;
}

int near_tc_launch(fda_plan_s* P, const float2* B, const float2* xt, float2* yt, int nrhs, int r0, int rc,
                   cudaStream_t s);

// wide batches on the tensor cores (near_form = 4): per pass of up to 64 right-hand sides, the off-block
// corrections by the CSR kernel (16 at a time), then one tensor-core pass over the matrices
static int near_tc_passes(fda_plan_s* P, const float2* B, const float2* cval, const float2* xt, float2* yt, int nrhs,
                          cudaStream_t s, int64_t* launches) {
  fda_tree_s* T = P->tree;
  for (int r0 = 0; r0 < nrhs; r0 += 64) {
    const int rc = std::min(64, nrhs - r0);
    for (int q0 = r0; q0 < r0 + rc; q0 += 16) {
      const int qc = std::min(16, r0 + rc - q0);
      k_near_corr<float2, 16><<<(unsigned)((T->N + 7) / 8), 256, 0, s>>>(P->corr_ptr.p, P->corr_col.p, cval, xt, yt,
                                                                         T->N, nrhs, q0, qc);
      FDA_LAUNCH_CHECK();
      ++*launches;
    }
    FDA_TRY(near_tc_launch(P, B, xt, yt, nrhs, r0, rc, s));
    ++*launches;
  }
  return FDA_OK;
}

template <typename C>
int near_stream(fda_plan_s* P, const C* B, const C* cval, const C* xt, C* yt, int nrhs, cudaStream_t s,
                int64_t* launches) {
  if (P->near_max_nr > NS_CONS) {
    set_error("near-field stream needs leaves of at most %d points (got %d)", NS_CONS, P->near_max_nr);
    return FDA_E_INVALID_ARG;
  }
  // the tensor-core form serves any batch width once chosen (the autotuner offers it from 16 right-hand sides)
  if constexpr (std::is_same<C, float2>::value)
    if (P->near_form == 4 && P->near_max_nr <= 64) return near_tc_passes(P, B, cval, xt, yt, nrhs, s, launches);
  // right-hand sides per pass over the matrix: 1, 4, or 16 for wide batches (each pass streams it once)
  if (nrhs == 1) {
    if constexpr (std::is_same<C, float2>::value)
      if (P->near_form == 2 && P->near_csep == 2 && P->xdup32.p)
        return near_stream_t<C, 1, true, 2>(P, B, cval, xt, yt, nrhs, s, launches);
    if constexpr (std::is_same<C, float2>::value)
      if (P->near_form == 3 && P->near_csep == 2)
        return near_stream_t<C, 1, true, 3>(P, B, cval, xt, yt, nrhs, s, launches);
    if (P->near_form == 1)
      return P->near_csep == 2 ? near_stream_t<C, 1, true, 1>(P, B, cval, xt, yt, nrhs, s, launches)
                               : near_stream_t<C, 1, false, 1>(P, B, cval, xt, yt, nrhs, s, launches);
    return P->near_csep == 2 ? near_stream_t<C, 1, true>(P, B, cval, xt, yt, nrhs, s, launches)
                             : near_stream_t<C, 1, false>(P, B, cval, xt, yt, nrhs, s, launches);
  }
  if constexpr (std::is_same<C, float2>::value)
    if (P->near_form == 2) {
      if (nrhs < 12 || P->near_wide == 0) return near_stream_t<C, 4, false, 2>(P, B, cval, xt, yt, nrhs, s, launches);
      return near_stream_t<C, 16, false, 2>(P, B, cval, xt, yt, nrhs, s, launches);
    }
  if (nrhs < 12 || P->near_wide == 0) return near_stream_t<C, 4, false>(P, B, cval, xt, yt, nrhs, s, launches);
  return near_stream_t<C, 16, false>(P, B, cval, xt, yt, nrhs, s, launches);
}

template int near_stream<float2>(fda_plan_s*, const float2*, const float2*, const float2*, float2*, int,
                                 cudaStream_t, int64_t*);
template int near_stream<double2>(fda_plan_s*, const double2*, const double2*, const double2*, double2*, int,
                                  cudaStream_t, int64_t*);

}  // namespace fda
