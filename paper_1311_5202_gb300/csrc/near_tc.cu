// Near field of wide batches (a6 with many right-hand sides) on the 5th-generation tensor cores.
//
// Each target leaf's near matrix B (nr rows x ncol columns, column-major complex, Eq. kcorrection's direct
// blocks with the in-block corrections folded in) meets up to 64 right-hand sides at once as one real GEMM
//   D[(r, q), n] += sum_k A[(r, q), k] Bt[n, k],   k = (column c, part p),
// with the densities as A and the matrix as Bt:
//   A[(r, 0), (c, 0)] = x_cr.re   A[(r, 0), (c, 1)] = x_cr.im
//   A[(r, 1), (c, 0)] = x_cr.im   A[(r, 1), (c, 1)] = -x_cr.re
//   Bt[n, (c, 0)] = B_nc.re       Bt[n, (c, 1)] = -B_nc.im
// so that D[(r, 0), n] and D[(r, 1), n] are the real and imaginary parts of (B x_r)_n. M = 128 real rows
// (64 right-hand sides), N = the leaf's rows rounded up to 16 (at most 64), K in chunks of 16 complex
// columns. Both operands are split into TF32 hi + lo parts and three products (hi hi + hi lo + lo hi) keep
// FP32 accuracy.
//
// Warp roles in a persistent CTA (one per SM, a contiguous range of target leaves):
//   - warp 8, one thread: streams the leaf's column-major matrix in chunks of 16 columns into a four-slot ring
//     (cp.async.bulk, completion on mbarriers), exactly as the FP32 near-field stream does;
//   - warps 0-7: per chunk, transpose the raw chunk into the K-major Bt image (hi, lo) and gather the
//     densities of the chunk's 16 columns for every right-hand side into the A image (hi, lo), both in the
//     canonical no-swizzle layout; thread 0 then issues the MMAs (accumulator in TMEM) and commits them to the
//     stage's mbarrier. Two stages: the next chunk is built while the tensor cores work on the current one;
//   - at a leaf's end, warps 0-7 read the accumulator with tcgen05.ld (warp w: lane quadrant w % 4, column
//     half w / 4) and add it into y (after the correction kernel stored its sums there).
//
// Every wait is bounded by 1 s of wall clock: a wait that gives up sets the error flag, the CTA stops taking
// work, still waits (bounded) for its own copies and MMAs in flight, and releases its TMEM.
#include "plan.cuh"
#include "tc_common.cuh"

namespace fda {

#define NTC_NT 288     // 8 builder warps + 1 producer warp
#define NTC_NB 256     // builder threads
#define NTC_CC 16      // complex columns per K chunk
#define NTC_KC 32      // real K per chunk
#define NTC_RAW 8192   // raw matrix bytes per ring slot: 16 columns x at most 64 rows x 8 bytes
#define NTC_RING 4
#define NTC_MAXR 64    // rows of a target leaf (N <= 64)
#define NTC_TCOLS 64   // TMEM columns (accumulator N <= 64)

struct NtcSmem {
  alignas(1024) float ahi[2][128 * NTC_KC];
  alignas(1024) float alo[2][128 * NTC_KC];
  alignas(1024) float bhi[2][NTC_MAXR * NTC_KC];
  alignas(1024) float blo[2][NTC_MAXR * NTC_KC];
  alignas(128) float2 raw[NTC_RING][NTC_RAW / 8];
  uint64_t rfull[NTC_RING], rempty[NTC_RING], mdone[2];
  uint32_t tmem;
  volatile int fail;
};

__device__ __forceinline__ void ntc_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NTC_NB) : "memory"); }

__device__ __forceinline__ void ntc_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void ntc_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void ntc_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// (value, hi, lo): hi = TF32(value), lo = value - hi
__device__ __forceinline__ void ntc_split(float v, float& hi, float& lo) {
  hi = tf32_round(v);
  lo = v - hi;
}

static __global__ void __launch_bounds__(NTC_NT, 1)
    k_near_tc(const int32_t* part, const NsMeta* meta, const int32_t* xcol, const float2* B, const float2* xt,
              float2* yt, int nrhs, int r0, int rc, int* err) {
  extern __shared__ unsigned char smem_raw[];
  NtcSmem& S = *reinterpret_cast<NtcSmem*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int u0 = part[blockIdx.x], u1 = part[blockIdx.x + 1];
  if (t == 0) {
    for (int i = 0; i < NTC_RING; ++i) {
      mbar_init(&S.rfull[i], 1);
      mbar_init(&S.rempty[i], NTC_NB / 32);
    }
    mbar_init(&S.mdone[0], 1);
    mbar_init(&S.mdone[1], 1);
    S.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(NTC_TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the A images start at zero: rows of right-hand sides beyond rc are never written again
  for (int i = t; i < 2 * 128 * NTC_KC / 4; i += NTC_NT) {
    reinterpret_cast<float4*>(&S.ahi[0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(&S.alo[0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;

  if (t >= NTC_NB) {
    // ---------------- producer: the leaves' matrices, 16 columns per ring slot
    if (t == NTC_NB) {
      int it = 0;
      bool ok = true;
      for (int u = u0; u < u1 && ok; ++u) {
        const NsMeta m = meta[u];
        const unsigned char* src = (const unsigned char*)(B + m.nb);
        for (int c0 = 0; c0 < m.ncol; c0 += NTC_CC) {
          const int cc = min(NTC_CC, m.ncol - c0);
          const int sl = it % NTC_RING;
          if (it >= NTC_RING && !mbar_wait(&S.rempty[sl], ((it / NTC_RING) - 1) & 1)) {
            atomicExch(err, 1);
            S.fail = 1;
            ok = false;
            break;
          }
          // c0 is a multiple of 16 and the matrix starts on 32 bytes: a 16-byte aligned source
          const uint32_t bytes = (uint32_t)(((int64_t)cc * m.nr * 8 + 15) & ~(int64_t)15);
          ntc_expect_tx(&S.rfull[sl], bytes);
          ntc_bulk(&S.raw[sl][0], src + (int64_t)c0 * m.nr * 8, bytes, &S.rfull[sl]);
          ++it;
        }
      }
      // the last fill of every slot has landed before the CTA's shared memory is released
      for (int j = max(0, it - NTC_RING); j < it; ++j) mbar_wait(&S.rfull[j % NTC_RING], (j / NTC_RING) & 1);
    }
    return;
  }

  // ---------------- builders, MMA issue (thread 0) and epilogue
  const uint32_t lbo = 128, sbo = (NTC_KC / 4) * 128;
  int it = 0;   // ring slot counter (same sequence as the producer)
  int kit = 0;  // chunk counter (stage = kit % 2)
  bool failed = false;
  for (int u = u0; u < u1 && !failed; ++u) {
    const NsMeta m = meta[u];
    const int nr = m.nr, ncol = m.ncol;
    if (ncol == 0) continue;
    const int N = max(16, (nr + 15) & ~15);
    const uint32_t idesc = idesc_tf32(128, N);
    for (int c0 = 0; c0 < ncol; c0 += NTC_CC) {
      const int cc = min(NTC_CC, ncol - c0);
      const int s = kit & 1;
      const int sl = it % NTC_RING;
      // densities of this chunk into registers first: their latency hides behind the transpose below
      float2 xv[4];
      int rr[4], cx[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = t + j * NTC_NB;  // (c, r) with r fastest: a column's right-hand sides are contiguous
        const int c = e >> 6, r = e & 63;
        rr[j] = r;
        cx[j] = c;
        xv[j] = make_float2(0.f, 0.f);
        if (c < cc && r < rc) xv[j] = xt[(int64_t)xcol[m.xb + c0 + c] * nrhs + r0 + r];
      }
      // stage s is free once the MMAs of chunk kit - 2 are done; the raw chunk has landed
      if (kit >= 2 && !mbar_wait(&S.mdone[s], ((kit >> 1) - 1) & 1)) S.fail = 1;
      if (!mbar_wait(&S.rfull[sl], (it / NTC_RING) & 1)) S.fail = 1;
      // Bt image: row n, K pair (2c, 2c + 1) = (B.re, -B.im); zeros past the leaf's rows and columns
      for (int e = t; e < N * NTC_CC; e += NTC_NB) {
        const int c = e / N, n = e - c * N;
        float2 b = make_float2(0.f, 0.f);
        if (n < nr && c < cc) b = S.raw[sl][c * nr + n];
        float h0, l0, h1, l1;
        ntc_split(b.x, h0, l0);
        ntc_split(-b.y, h1, l1);
        const uint32_t off = kmaj_off(n, 2 * c, NTC_KC) / 4;
        *reinterpret_cast<float2*>(&S.bhi[s][off]) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(&S.blo[s][off]) = make_float2(l0, l1);
      }
      __syncwarp();
      if (lane == 0) ntc_arrive(&S.rempty[sl]);  // this warp is done with the raw slot
      // A image: rows (r, 0) = (x.re, x.im) and (r, 1) = (x.im, -x.re) for the chunk's columns
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = rr[j], c = cx[j];
        if (r >= rc) continue;
        float a0, a1, b0, b1, c0h, c0l;
        ntc_split(xv[j].x, a0, b0);     // x.re
        ntc_split(xv[j].y, a1, b1);     // x.im
        ntc_split(-xv[j].x, c0h, c0l);  // -x.re
        const uint32_t o0 = kmaj_off(2 * r, 2 * c, NTC_KC) / 4, o1 = kmaj_off(2 * r + 1, 2 * c, NTC_KC) / 4;
        *reinterpret_cast<float2*>(&S.ahi[s][o0]) = make_float2(a0, a1);
        *reinterpret_cast<float2*>(&S.alo[s][o0]) = make_float2(b0, b1);
        *reinterpret_cast<float2*>(&S.ahi[s][o1]) = make_float2(a1, c0h);
        *reinterpret_cast<float2*>(&S.alo[s][o1]) = make_float2(b1, c0l);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ntc_sync();
      if (S.fail) {
        failed = true;
        break;
      }
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int s8 = 0; s8 < NTC_KC / 8; ++s8) {
          if (s8 * 8 >= 2 * cc) break;  // K steps past the chunk's columns hold only zeros
          const uint64_t ad = smem_desc(smem_u32(S.ahi[s]) + s8 * 256, lbo, sbo);
          const uint64_t adl = smem_desc(smem_u32(S.alo[s]) + s8 * 256, lbo, sbo);
          const uint64_t bd = smem_desc(smem_u32(S.bhi[s]) + s8 * 256, lbo, sbo);
          const uint64_t bdl = smem_desc(smem_u32(S.blo[s]) + s8 * 256, lbo, sbo);
          const int acc = (c0 > 0 || s8 > 0) ? 1 : 0;
          tc_mma(tmem, adl, bd, idesc, acc);  // the small products first, then hi * hi
          tc_mma(tmem, ad, bdl, idesc, 1);
          tc_mma(tmem, ad, bd, idesc, 1);
        }
        tc_commit(&S.mdone[s]);
      }
      ++it;
      ++kit;
    }
    if (failed) break;
    // leaf end: the last chunk's MMAs are done, the accumulator goes into y
    if (!mbar_wait(&S.mdone[(kit - 1) & 1], ((kit - 1) >> 1) & 1)) S.fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ntc_sync();
    if (S.fail) {
      failed = true;
      break;
    }
    const int q4 = w & 3, h = w >> 2;
    const int r = 16 * q4 + (lane >> 1), part = lane & 1;
    for (int cb = 32 * h; cb < min(32 * h + 32, N); cb += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)cb, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float other = __shfl_xor_sync(0xffffffffu, v[j], 1);
        const int n = cb + j;
        if (part == 0 && n < nr && r < rc) {
          float2* yp = yt + (m.tb + n) * nrhs + r0 + r;
          const float2 y0 = *yp;
          *yp = make_float2(y0.x + v[j], y0.y + other);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ntc_sync();  // every TMEM read is done before the next leaf's first MMA overwrites the accumulator
  }
  // MMAs still in flight (after a wait that gave up) finish before the TMEM is released
  if (failed) atomicExch(err, 1);
  if (t == 0 && kit > 0) mbar_wait(&S.mdone[(kit - 1) & 1], ((kit - 1) >> 1) & 1);
  if (t == 0 && kit > 1) mbar_wait(&S.mdone[kit & 1], ((kit - 2) >> 1) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  ntc_sync();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NTC_TCOLS));
  }
}

// y (tree order, FP32) += near-field products of right-hand sides r0 .. r0 + rc - 1 (rc <= 64), one CTA per SM
// over the plan's one-CTA-per-SM partition of the target leaves; the caller has run the correction kernel
int near_tc_launch(fda_plan_s* P, const float2* B, const float2* xt, float2* yt, int nrhs, int r0, int rc,
                   cudaStream_t s) {
  if (rc < 1 || rc > 64 || P->near_max_nr > NTC_MAXR || P->near_grid_ov[1] <= 0) {
    set_error("tensor-core near field: %d right-hand sides per pass, leaves of at most %d rows", rc, NTC_MAXR);
    return FDA_E_INVALID_ARG;
  }
  const size_t smem = sizeof(NtcSmem) + 1024;
  static bool attr = false;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_near_tc<<<(unsigned)P->near_grid_ov[1], NTC_NT, smem, s>>>(P->near_part_ov[1].p, P->near_meta.p,
                                                               P->near_xcol.p, B, xt, yt, nrhs, r0, rc,
                                                               P->tc_err.p);
  FDA_LAUNCH_CHECK();
  return FDA_OK;
}

}  // namespace fda
