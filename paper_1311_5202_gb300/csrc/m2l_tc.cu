// M2L on the 5th-generation tensor cores (tcgen05, kind::tf32, accumulators in TMEM).
//
// A complex product y = A x (A: M x K, column-major complex) is one real GEMM on interleaved (re, im)
// storage: with A^ the 2x2 real block expansion [[Ar, -Ai], [Ai, Ar]] of every entry, rows 2i / 2i+1 of
// A^ x^ are the real / imaginary parts of y_i, and x^ is the complex vector read as 2K reals. Each CTA
// computes one 128-row tile of A^ (64 complex rows) against up to 64 gathered columns (pairs x RHS):
// the A^ tile is expanded on the fly, both operands are staged in shared memory in the canonical K-major
// layout without swizzle (8-row x 16-byte core matrices), one thread issues tcgen05.mma (K = 8 per
// instruction) and commits to an mbarrier, and the accumulator (128 lanes x 64 FP32 columns) is read back
// with tcgen05.ld and scattered with atomics. With split = 1 every operand is split into TF32 hi + lo and
// three products (hi hi + hi lo + lo hi) keep FP32 accuracy. Every wait is bounded: a wait that gives up
// sets an error flag, and the kernel still releases its TMEM.
#include <cuda.h>

#include "plan.cuh"
#include "tc_common.cuh"

#include <vector>

namespace fda {

#define TC_M 128       // real rows per tile (64 complex rows)
#define TC_N 64        // real GEMM columns per tile (pairs x RHS)
#define TC_KC 32       // real K per stage (16 complex)
#define TC_NT 128      // threads per CTA (4 warps: one TMEM lane quadrant each)
#define TC_MT 4      // row tiles per CTA (up to 256 complex rows)

// Shared memory per pipeline buffer: A^ tiles (TC_MT x 128 x KC), B tile (64 x KC), hi and (split) lo parts
template <int KC, int MTC, int SPLIT>
struct TcBuf {
  alignas(128) float a_hi[MTC][TC_M * KC];
  alignas(128) float a_lo[MTC][SPLIT ? TC_M * KC : 4];
  alignas(128) float b_hi[TC_N * KC];
  alignas(128) float b_lo[SPLIT ? TC_N * KC : 4];
};
template <int KC, int MTC, int SPLIT>
struct TcSmem {
  TcBuf<KC, MTC, SPLIT> buf[2];
  alignas(8) uint64_t bar[2];
  uint32_t tmem;
  int64_t sbase[TC_N], dbase[TC_N];
  int srr[TC_N];
};

// Grouped gather-GEMM-scatter on the tensor cores; same units and modes as the FMA k_m2l
// (0: coef_out -> coef_in add, 1: coef_out -> mid store, 2: mid -> coef_in add). A unit covers output rows
// [m0, min(M, m0 + 256)); its gathered columns are staged once per K-chunk and reused by every row tile.
// Two shared-memory buffers: the loads of chunk k+1 overlap the MMAs of chunk k.
template <int SPLIT, int MTC>
static __global__ void __launch_bounds__(TC_NT) k_m2l_tc(const GemmUnit* units, const float2* poolK,
                                                         const float2* poolLR, const int64_t* psrc,
                                                         const int64_t* ptgt, const int64_t* pmid,
                                                         const float2* cout, float2* cin, float2* mid, int nrhs,
                                                         int64_t ldc, int64_t ldm, int* err) {
  constexpr int KC = SPLIT ? 16 : 32;  // real K per chunk
  extern __shared__ unsigned char smem_raw[];
  typedef TcSmem<KC, MTC, SPLIT> Sm;
  Sm& S = *reinterpret_cast<Sm*>((((uintptr_t)smem_raw) + 127) & ~(uintptr_t)127);
  const GemmUnit U = units[blockIdx.x];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const float2* A = (U.mode == 0 ? poolK : poolLR) + U.a_off;
  const float2* X = (U.mode == 2) ? mid : cout;
  const int64_t lds = (U.mode == 2) ? ldm : ldc, ldd = (U.mode == 1) ? ldm : ldc;  // right-hand-side strides
  const int rows = min(U.M - U.m0, 64 * MTC);  // complex rows of this unit
  const int MT = (rows + 63) / 64;
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(TC_N * (MTC < 2 ? 2 : MTC)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;
  const int ncols = U.p_count * nrhs;
  const int Kr = 2 * U.K;
  const int nk = (Kr + KC - 1) / KC;
  uint32_t ph[2] = {0, 0};
  bool ok = true;
  constexpr uint32_t IDESC = idesc_tf32(TC_M, TC_N);

  auto load_chunk = [&](int kc, TcBuf<KC, MTC, SPLIT>& B) {
    const int k0 = kc * KC;
    for (int mt = 0; mt < MT; ++mt)
      for (int q = t; q < 64 * (KC / 2); q += TC_NT) {
        int i = q & 63, j = q >> 6;
        int gi = U.m0 + 64 * mt + i, gj = k0 / 2 + j;
        float2 a = (gi < U.M && gj < U.K) ? A[gi + (int64_t)gj * U.M] : make_float2(0.f, 0.f);
        float v[4] = {a.x, -a.y, a.y, a.x};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          uint32_t off = kmaj_off(2 * i + (u >> 1), 2 * j + (u & 1), KC) / 4;
          float hi = tf32_round(v[u]);
          B.a_hi[mt][off] = hi;
          if (SPLIT) B.a_lo[mt][off] = tf32_round(v[u] - hi);
        }
      }
    for (int q = t; q < TC_N * (KC / 2); q += TC_NT) {
      int j = q % (KC / 2), n = q / (KC / 2);
      int gj = k0 / 2 + j;
      float2 x = (S.sbase[n] >= 0 && gj < U.K) ? X[(int64_t)S.srr[n] * lds + S.sbase[n] + gj] : make_float2(0.f, 0.f);
      float v[2] = {x.x, x.y};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        uint32_t off = kmaj_off(n, 2 * j + u, KC) / 4;
        float hi = tf32_round(v[u]);
        B.b_hi[off] = hi;
        if (SPLIT) B.b_lo[off] = tf32_round(v[u] - hi);
      }
    }
  };
  auto wait_uniform = [&](int b) {
    bool mine = mbar_wait(&S.bar[b], ph[b]);
    bool all = __syncthreads_and(mine ? 1 : 0) != 0;
    if (!all) {
      if (t == 0) atomicExch(err, 1);
      mbar_wait(&S.bar[b], ph[b]);  // second bounded wait for the MMAs still in flight
    }
    ph[b] ^= 1;
    return all;
  };

  for (int c0 = 0; c0 < ncols && ok; c0 += TC_N) {
    if (t < TC_N) {
      int c = c0 + t;
      if (c < ncols) {
        int p = c / nrhs, rr = c - p * nrhs;
        int64_t pi = U.p_begin + p;
        S.sbase[t] = (U.mode == 2) ? pmid[pi] : psrc[pi];
        S.dbase[t] = (U.mode == 1) ? pmid[pi] : ptgt[pi];
        S.srr[t] = rr;
      } else {
        S.sbase[t] = -1;
        S.dbase[t] = -1;
        S.srr[t] = 0;
      }
    }
    __syncthreads();
    load_chunk(0, S.buf[0]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    bool pending[2] = {false, false};
    for (int kc = 0; kc < nk; ++kc) {
      const int b = kc & 1;
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t lbo = 128, sbo = (KC / 4) * 128;
        for (int mt = 0; mt < MT; ++mt) {
          const uint32_t dt = tmem + 64 * mt;
#pragma unroll
          for (int s8 = 0; s8 < KC / 8; ++s8) {
            uint32_t ks = s8 * 256;
            uint64_t ah = smem_desc(smem_u32(S.buf[b].a_hi[mt]) + ks, lbo, sbo);
            uint64_t bh = smem_desc(smem_u32(S.buf[b].b_hi) + ks, lbo, sbo);
            tc_mma(dt, ah, bh, IDESC, (kc > 0 || s8 > 0) ? 1 : 0);
            if (SPLIT) {
              uint64_t al = smem_desc(smem_u32(S.buf[b].a_lo[mt]) + ks, lbo, sbo);
              uint64_t bl = smem_desc(smem_u32(S.buf[b].b_lo) + ks, lbo, sbo);
              tc_mma(dt, ah, bl, IDESC, 1);
              tc_mma(dt, al, bh, IDESC, 1);
            }
          }
        }
        tc_commit(&S.bar[b]);
      }
      pending[b] = true;
      if (kc + 1 < nk) {
        const int nb = b ^ 1;
        if (pending[nb]) {  // chunk kc-1 used buffer nb: its MMAs must finish before it is overwritten
          ok = wait_uniform(nb);
          pending[nb] = false;
          if (!ok) break;
        }
        load_chunk(kc + 1, S.buf[nb]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncthreads();
    }
    for (int b = 0; b < 2; ++b)
      if (pending[b]) {
        bool r = wait_uniform(b);
        ok = ok && r;
      }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int row = 32 * w + lane;  // real row within a tile
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        const int ci = U.m0 + 64 * mt + (row >> 1);
        const int part = row & 1;
#pragma unroll
        for (int h = 0; h < TC_N / 32; ++h) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * w) << 16) + 64 * mt + 32 * h, v);
          if (ci < U.M) {
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              int n = 32 * h + q;
              if (S.dbase[n] < 0) continue;
              int64_t d = (int64_t)S.srr[n] * ldd + S.dbase[n] + ci;
              if (U.mode == 1)
                ((float*)(mid + d))[part] = v[q];
              else
                atomicAdd(((float*)(cin + d)) + part, v[q]);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N * (MTC < 2 ? 2 : MTC)));
  }
}

template <int SPLIT, int MTC>
static size_t tc_smem() {
  return sizeof(TcSmem<SPLIT ? 16 : 32, MTC, SPLIT>) + 128;
}

template <int SPLIT, int MTC>
static int tc_launch(const GemmUnit* units, size_t nunits, const float2* poolK, const float2* poolLR,
                     const int64_t* psrc, const int64_t* ptgt, const int64_t* pmid, const float2* cout, float2* cin,
                     float2* mid, int nrhs, int64_t ldc, int64_t ldm, int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_m2l_tc<SPLIT, MTC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem<SPLIT, MTC>()));
    attr = true;
  }
  for (size_t u0 = 0; u0 < nunits; u0 += 65535) {
    unsigned n = (unsigned)std::min<size_t>(65535, nunits - u0);
    k_m2l_tc<SPLIT, MTC><<<n, TC_NT, tc_smem<SPLIT, MTC>(), s>>>(units + u0, poolK, poolLR, psrc, ptgt, pmid, cout,
                                                                 cin, mid, nrhs, ldc, ldm, err);
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// max_rows: the largest number of complex output rows any unit of this launch covers (<= 256)
int m2l_tc_launch(const GemmUnit* units, size_t nunits, const float2* poolK, const float2* poolLR,
                  const int64_t* psrc, const int64_t* ptgt, const int64_t* pmid, const float2* cout, float2* cin,
                  float2* mid, int nrhs, int64_t ldc, int64_t ldm, int split, int max_rows, int* err, cudaStream_t s) {
  int mt = (max_rows + 63) / 64;
#define TCL(S_, M_) \
  return tc_launch<S_, M_>(units, nunits, poolK, poolLR, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s)
  if (split) {
    if (mt <= 1) TCL(1, 1);
    if (mt <= 2) TCL(1, 2);
    TCL(1, 4);
  } else {
    if (mt <= 1) TCL(0, 1);
    if (mt <= 2) TCL(0, 2);
    TCL(0, 4);
  }
#undef TCL
}


// ================================================================== TF32 form with pre-expanded operators
// Each operator (K~, or U^ and V^) is expanded once at plan time into the exact shared-memory image the
// MMA reads: per 128-row tile and per 32-wide real K chunk, the canonical K-major no-swizzle layout
// (8-row groups of 1 KB), rounded to TF32, with only the 8-row groups that hold rows stored. A unit is
// one operator with up to 128 pairs and covers all its output rows (up to MTC tiles, accumulators in
// TMEM). Per K chunk, one thread copies the operator tiles with cp.async.bulk (completion on an
// mbarrier with transaction bytes) while all threads gather the pairs' source coefficients with 16-byte
// cp.async, two complex values per copy (zero fill past K; every coefficient vector starts 16-byte aligned
// because ranks are even and intermediates padded to even length); NST chunks are in flight. The MMA issuer commits each chunk to a
// per-stage mbarrier that frees its buffers. Epilogue: warp w reads TMEM lane quadrant w % 4 and half of
// the columns; lanes hold consecutive real rows, and after a lane-pair exchange every lane owns one complex
// value, so a warp updates 16 consecutive complex coefficients of each of two columns per instruction
// (8-byte atomics, or stores into the low-rank intermediate).

__device__ __forceinline__ int tc3_ng(int M, int mt) { return (min(128, 2 * M - 128 * mt) + 7) / 8; }

static __global__ void k_tc3_image(const TcImgJob* jobs, float* img) {
  const TcImgJob J = jobs[blockIdx.y];
  const int MT = (2 * J.M + 127) / 128, nk = (2 * J.K + 31) / 32;
  const int64_t full_tile = (int64_t)nk * 16 * 256;
  const int last_ng = tc3_ng(J.M, MT - 1);
  const int64_t total = (int64_t)(MT - 1) * full_tile + (int64_t)nk * last_ng * 256;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int mt = (int)(q / full_tile < (int64_t)(MT - 1) ? q / full_tile : (int64_t)(MT - 1));
    const int64_t rem = q - mt * full_tile;
    const int ng = (mt < MT - 1) ? 16 : last_ng;
    const int kc = (int)(rem / (ng * 256));
    const int o = (int)(rem - (int64_t)kc * ng * 256);
    const int grp = o >> 8, within = o & 255;
    const int row = grp * 8 + ((within & 31) >> 2);
    const int kk = (within >> 5) * 4 + (within & 3);
    const int j = 128 * mt + row, kr = 32 * kc + kk;
    const int i = j >> 1, kx = kr >> 1;
    float val = 0.f, vlo = 0.f;
    if (i < J.M && kx < J.K) {
      const double2 a = J.trans ? J.src[kx + (int64_t)i * J.ld] : J.src[i + (int64_t)kx * J.ld];
      const double v = (j & 1) == 0 ? ((kr & 1) == 0 ? a.x : -a.y) : ((kr & 1) == 0 ? a.y : a.x);
      val = tf32_round((float)v);
      vlo = tf32_round((float)(v - (double)val));
    }
    img[J.img_off + q] = val;
    if (J.split) img[J.img_off + total + q] = vlo;  // the remainder image follows the TF32 image
  }
}

int tc3_build_images(const std::vector<TcImgJob>& jobs, float* img) {
  if (jobs.empty()) return FDA_OK;
  DBuf<TcImgJob> dj;
  FDA_TRY(dj.upload(jobs));
  for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
    unsigned nb = (unsigned)std::min<size_t>(65535, jobs.size() - b0);
    k_tc3_image<<<dim3(16, nb), 256>>>(dj.p + b0, img);
    FDA_LAUNCH_CHECK();
  }
  FDA_CUDA(cudaDeviceSynchronize());
  return FDA_OK;
}

__device__ __forceinline__ void tc3_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tc3_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc3_cp8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void tc3_cp16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void tc3_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tc3_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

#define TC3_KC 32
#define TC3_NT 256

// complex-pair epilogue helper: lanes 2i (real part) and 2i+1 (imaginary part) hold row i of columns
// c and c + 1; after one exchange the even lane owns column c and the odd lane column c + 1, each as a
// complex value (one 8-byte update per lane instead of two 4-byte ones)
__device__ __forceinline__ float2 tc_pair(const float* v, int c, int part) {
  const float send = part == 0 ? v[c + 1] : v[c];
  const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
  return part == 0 ? make_float2(v[c], recv) : make_float2(recv, v[c + 1]);
}

template <int MTC, int N, int NST, int SPLIT = 0>
struct Tc3Smem {
  alignas(1024) float a[NST][MTC][128 * TC3_KC];
  alignas(1024) float b[NST][N * TC3_KC];
  // 3xTF32: the operator remainders and the remainders of the gathered coefficients
  alignas(1024) float alo[SPLIT ? NST : 1][SPLIT ? MTC : 1][SPLIT ? 128 * TC3_KC : 256];
  alignas(1024) float blo[SPLIT ? NST : 1][SPLIT ? N * TC3_KC : 256];
  alignas(8) uint64_t afull[NST];
  uint64_t mdone[NST];
  uint32_t tmem;
  int64_t sbase[N], dbase[N];
  int srr[N];
};

// One CTA per unit (operator, up to 128 pairs); all its output rows (up to MTC tiles) in TMEM. Per K chunk,
// thread 0 copies the operator tiles with cp.async.bulk while all threads gather the pairs' coefficients
// with 16-byte cp.async (two complex values; 8-byte copies for a source off a 16-byte boundary); NST chunks
// in flight.
template <int MTC, int N, int NST, int BULK, int SPLIT>
static __global__ void __launch_bounds__(TC3_NT) k_m2l_tc3(const GemmUnit* units, const float* img,
                                                          const int64_t* psrc, const int64_t* ptgt,
                                                          const int64_t* pmid, const float2* cout, float2* cin,
                                                          float2* mid, int nrhs, int64_t ldc, int64_t ldm, int* err) {
  typedef Tc3Smem<MTC, N, NST, SPLIT> Sm;
  extern __shared__ unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  // TMEM allocations are powers of two of at least 32 columns
  constexpr int TCOLS = MTC * N <= 32 ? 32 : MTC * N <= 64 ? 64 : MTC * N <= 128 ? 128 : MTC * N <= 256 ? 256 : 512;
  constexpr uint32_t IDESC = idesc_tf32(128, N);
  // refill distance: chunk kc + D is issued at step kc into the stage that served chunk kc + D - NST
  constexpr int D = NST - 1;
  const GemmUnit U = units[blockIdx.x];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const float2* X = (U.mode == 2) ? mid : cout;
  const int64_t lds = (U.mode == 2) ? ldm : ldc, ldd = (U.mode == 1) ? ldm : ldc;  // right-hand-side strides
  const int MT = min(MTC, (2 * U.M + 127) / 128);
  const int nk = (2 * U.K + TC3_KC - 1) / TC3_KC;
  const float* A = img + U.a_off;
  const float* Alo = A + (SPLIT ? tc3_image_floats(U.M, U.K) : 0);  // remainder image (3xTF32)
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&S.afull[s], 1);
      mbar_init(&S.mdone[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;
  uint32_t ph_a[NST], ph_m[NST];
#pragma unroll
  for (int s = 0; s < NST; ++s) ph_a[s] = ph_m[s] = 0;
  bool ok = true;
  // every thread takes the same branch: the wait result is made uniform across the CTA
  auto wait_mdone = [&](int s) {
    bool mine = mbar_wait(&S.mdone[s], ph_m[s]);
    bool all = __syncthreads_and(mine ? 1 : 0) != 0;
    if (!all) {
      if (t == 0) atomicExch(err, 1);
      mbar_wait(&S.mdone[s], ph_m[s]);  // second bounded wait for MMAs still in flight
    }
    ph_m[s] ^= 1;
    return all;
  };
  auto issue = [&](int kc) {
    const int s = kc % NST;
    if (t == 0) {
      uint32_t bytes = 0;
      for (int mt = 0; mt < MT; ++mt) bytes += (uint32_t)tc3_ng(U.M, mt) * 1024u;
      tc3_expect_tx(&S.afull[s], SPLIT ? 2 * bytes : bytes);
      for (int mt = 0; mt < MT; ++mt) {
        const int ng = tc3_ng(U.M, mt);
        const int64_t o = (int64_t)16 * mt * nk * 256 + (int64_t)kc * ng * 256;
        tc3_bulk(S.a[s][mt], A + o, (uint32_t)ng * 1024u, &S.afull[s]);
        if (SPLIT) tc3_bulk(S.alo[s][mt], Alo + o, (uint32_t)ng * 1024u, &S.afull[s]);
      }
    }
    const uint32_t bbase = smem_u32(S.b[s]);
    // two complex values (16 bytes, one K-major core row segment) per copy: lane = (column n mod 8, pair
    // of K indices); four lanes read 64 contiguous bytes of a column
    for (int r = w; r < (N / 8) * 2; r += TC3_NT / 32) {
      const int n = (r >> 1) * 8 + (lane >> 2), j = (r & 1) * 8 + 2 * (lane & 3);
      if (S.sbase[n] < 0) continue;  // unused column: its results are never read
      const int gj = kc * (TC3_KC / 2) + j;
      const uint32_t dst = bbase + kmaj_off(n, 2 * j, TC3_KC);
      const float2* src = gj < U.K ? X + (int64_t)S.srr[n] * lds + S.sbase[n] + gj : X;
      const uint32_t nb = gj + 1 < U.K ? 16u : (gj < U.K ? 8u : 0u);  // the rest is zero-filled
      if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        tc3_cp16(dst, src, nb);
      } else {  // odd coefficient offset: two 8-byte copies
        tc3_cp8(dst, src, nb >= 8 ? 8u : 0u);
        tc3_cp8(dst + 8, nb == 16 ? src + 1 : X, nb == 16 ? 8u : 0u);
      }
    }
    tc3_commit_group();
  };

  const int ncols = U.p_count * nrhs;
  for (int c0 = 0; c0 < ncols && ok; c0 += N) {
    if (t < N) {
      const int c = c0 + t;
      if (c < ncols) {
        const int p = c / nrhs, rr = c - p * nrhs;
        const int64_t pi = U.p_begin + p;
        S.sbase[t] = (U.mode == 2) ? pmid[pi] : psrc[pi];
        S.dbase[t] = (U.mode == 1) ? pmid[pi] : ptgt[pi];
        S.srr[t] = rr;
      } else {
        S.sbase[t] = -1;
        S.dbase[t] = -1;
        S.srr[t] = 0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < D; ++j) {
      if (j < nk)
        issue(j);
      else
        tc3_commit_group();
    }
    for (int kc = 0; kc < nk; ++kc) {
      const int j = kc + D;
      if (j < nk) {
        if (j >= NST) ok = wait_mdone(j % NST) && ok;  // MMAs of chunk j - NST (<= kc - 1) released this stage
        issue(j);
      } else {
        tc3_commit_group();
      }
      tc3_wait_group<D>();  // this thread's copies of chunk kc have landed
      if (SPLIT) {
        // every thread splits the segments it gathered into a TF32 part (in place) and its remainder
        const int s = kc % NST;
        for (int r = w; r < (N / 8) * 2; r += TC3_NT / 32) {
          const int n = (r >> 1) * 8 + (lane >> 2), j = (r & 1) * 8 + 2 * (lane & 3);
          if (S.sbase[n] < 0) continue;
          const uint32_t off = kmaj_off(n, 2 * j, TC3_KC) / 4;
          float4 v = *reinterpret_cast<float4*>(&S.b[s][off]);
          float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
          *reinterpret_cast<float4*>(&S.b[s][off]) = h;
          *reinterpret_cast<float4*>(&S.blo[s][off]) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (t == 0) {
        const int s = kc % NST;
        if (!mbar_wait(&S.afull[s], ph_a[s])) atomicExch(err, 1);
        ph_a[s] ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t lbo = 128, sbo = (TC3_KC / 4) * 128;
        for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
          for (int s8 = 0; s8 < TC3_KC / 8; ++s8) {
            if (kc * TC3_KC + s8 * 8 >= 2 * U.K) break;  // K steps past the operator hold only zeros
            const uint64_t ad = smem_desc(smem_u32(S.a[s][mt]) + s8 * 256, lbo, sbo);
            const uint64_t bd = smem_desc(smem_u32(S.b[s]) + s8 * 256, lbo, sbo);
            const int acc = (kc > 0 || s8 > 0) ? 1 : 0;
            if (SPLIT) {  // the small products first, then hi * hi
              const uint64_t adl = smem_desc(smem_u32(S.alo[s][mt]) + s8 * 256, lbo, sbo);
              const uint64_t bdl = smem_desc(smem_u32(S.blo[s]) + s8 * 256, lbo, sbo);
              tc_mma(tmem + N * mt, adl, bd, IDESC, acc);
              tc_mma(tmem + N * mt, ad, bdl, IDESC, 1);
              tc_mma(tmem + N * mt, ad, bd, IDESC, 1);
            } else {
              tc_mma(tmem + N * mt, ad, bd, IDESC, acc);
            }
          }
        }
        tc_commit(&S.mdone[s]);
      }
    }
    for (int c = max(0, nk - NST); c < nk; ++c) ok = wait_mdone(c % NST) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (BULK && U.mode != 1 && (U.M & 1) == 0) {  // bulk reductions move whole 16-byte granules
      // Bulk-reduction epilogue: the accumulators go through shared memory, 16 columns at a time in two
      // alternating buffers aliased on the operator tiles (every MMA of this column block has completed and no
      // copy writes them before the next block starts), and each column (a pair's complex output vector,
      // U.M values) is added to its target with one cp.reduce.async.bulk; the copy engine performs the adds
      // while the CTA moves on. Warps 0-3 read the even row tiles, warps 4-7 the odd ones (TMEM lane
      // quadrant w % 4).
      float* stg = &S.a[0][0][0];
      const int RT = 128 * MT;  // staged real rows per column
      const int q4 = w & 3;
      for (int cg = 0; cg < N / 16; ++cg) {
        float* sb = stg + (cg & 1) * 16 * RT;
        if (t < 16) bulk_wait_read<1>();  // the reductions that read this buffer two groups ago are done
        __syncthreads();
        if (ok) {
          for (int mt = w >> 2; mt < MT; mt += 2) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(N * mt + 16 * cg), v);
            const int row = 128 * mt + 32 * q4 + lane;
#pragma unroll
            for (int c = 0; c < 16; ++c) sb[c * RT + row] = v[c];
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t < 16) {
          const int n = 16 * cg + t;
          const int64_t db = S.dbase[n];
          if (ok && db >= 0) {
            float2* dst = cin + (int64_t)S.srr[n] * ldd + db;
            if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)
              bulk_reduce_add(dst, sb + t * RT, 8u * (uint32_t)U.M);
            else
              atomicExch(err, 2);  // a target off a 16-byte boundary (the plan never makes one): reported, skipped
          }
          bulk_commit();
        }
      }
      if (t < 16) bulk_wait_read<0>();
    } else {
    // columns per warp: half of the tile for N >= 64; the whole tile (warps 0-3 only) for N = 32
    constexpr int CPW = N >= 64 ? N / 2 : N;
    if (ok && (N >= 64 || w < 4)) {
      const int q4 = w & 3, half = N >= 64 ? (w >> 2) : 0;
      const int row = 32 * q4 + lane;  // real row within a tile
      const int part = row & 1;
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        const int ci = 64 * mt + (row >> 1);
#pragma unroll 1
        for (int h = 0; h < CPW / 32; ++h) {
          const int col0 = half * CPW + 32 * h;
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(N * mt + col0), v);
#pragma unroll
          for (int q = 0; q < 32; q += 2) {
            const float2 val = tc_pair(v, q, part);
            const int n = col0 + q + part;
            const int64_t db = S.dbase[n];
            if (db < 0 || ci >= U.M) continue;
            const int64_t d = (int64_t)S.srr[n] * ldd + db + ci;
            if (U.mode == 1)
              mid[d] = val;
            else
              atomicAdd(cin + d, val);
          }
        }
      }
    }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

template <int MTC, int N, int NST, int BULK, int SPLIT = 0>
static int tc3_launch_t(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc,
                        const int64_t* ptgt, const int64_t* pmid, const float2* cout, float2* cin, float2* mid,
                        int nrhs, int64_t ldc, int64_t ldm, int* err, cudaStream_t s) {
  const size_t smem = sizeof(Tc3Smem<MTC, N, NST, SPLIT>) + 1024;
  static bool attr = false;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_m2l_tc3<MTC, N, NST, BULK, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = true;
  }
  for (size_t u0 = 0; u0 < nunits; u0 += 65535) {
    unsigned n = (unsigned)std::min<size_t>(65535, nunits - u0);
    k_m2l_tc3<MTC, N, NST, BULK, SPLIT><<<n, TC3_NT, smem, s>>>(units + u0, img, psrc, ptgt, pmid, cout, cin, mid,
                                                                nrhs, ldc, ldm, err);
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// max_mt: the largest number of 128-row tiles of any unit of this launch (1..4); max_k: the largest complex
// K. Launches whose K fits two 32-wide real chunks (the U^ stage of low-rank pairs) gain little from double
// buffering and run single-stage, smaller CTAs, several per SM. shape 0 is the default tile shape of each
// class, shapes 1 to 3 alternatives (other column width or stage count) that the autotuner may pick.
int m2l_tc3_launch(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc, const int64_t* ptgt,
                   const int64_t* pmid, const float2* cout, float2* cin, float2* mid, int nrhs, int64_t ldc,
                   int64_t ldm, int max_mt, int max_k, int* err, cudaStream_t s, int shape) {
  if (max_mt < 1 || max_mt > 4) {
    set_error("tensor-core M2L supports at most 256 complex output rows (got %d tiles)", max_mt);
    return FDA_E_INVALID_ARG;
  }
  if (nunits == 0) return FDA_OK;
  if (shape == 6 || shape == 7) {  // 3xTF32 from the TF32 and remainder images, single stage: 6 atomics, 7 bulk
#define TC3S(M_, N_, B_) \
  return tc3_launch_t<M_, N_, 1, B_, 1>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s)
    if (shape == 6) {
      if (max_mt == 1) TC3S(1, 128, 0);
      if (max_mt == 2) TC3S(2, 64, 0);
      TC3S(4, 64, 0);
    }
    if (max_mt == 1) TC3S(1, 128, 1);
    if (max_mt == 2) TC3S(2, 64, 1);
    TC3S(4, 64, 1);
#undef TC3S
  }
  if (shape == 8) {  // bulk reductions, single stage, 32 columns and exactly the rows needed: most CTAs per SM
#define TC3N(M_) \
  return tc3_launch_t<M_, 32, 1, 1>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s)
    if (max_mt == 1) TC3N(1);
    if (max_mt == 2) TC3N(2);
    if (max_mt == 3) TC3N(3);
    TC3N(4);
#undef TC3N
  }
  if (shape == 4 || shape == 5) {  // bulk-reduction epilogue: default shape (4) or single-stage (5)
#define TC3B(M_, N_, S_) \
  return tc3_launch_t<M_, N_, S_, 1>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s)
    const bool short_k = max_k > 0 && 2 * max_k <= 2 * TC3_KC;
    if (shape == 5 || short_k) {
      if (max_mt == 1) TC3B(1, 128, 1);
      if (max_mt == 2) TC3B(2, 64, 1);
      TC3B(4, 64, 1);
    }
    if (max_mt == 1) TC3B(1, 128, 3);
    if (max_mt == 2) TC3B(2, 128, 2);
    TC3B(4, 64, 2);
#undef TC3B
  }
#define TC3L(M_, N_, S_) \
  return tc3_launch_t<M_, N_, S_, 0>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s)
  const bool alt = shape == 1;
  if (shape == 2) {  // single-stage
    if (max_mt == 1) TC3L(1, 128, 1);
    if (max_mt == 2) TC3L(2, 64, 1);
    TC3L(4, 64, 1);
  }
  if (shape == 3) {  // single-stage, narrow: the most CTAs per SM (TMEM and shared memory)
    if (max_mt == 1) TC3L(1, 64, 1);
    if (max_mt == 2) TC3L(2, 32, 1);
    TC3L(4, 32, 1);
  }
  if (max_k > 0 && 2 * max_k <= 2 * TC3_KC) {
    if (max_mt == 1) {
      if (alt) TC3L(1, 64, 1);
      TC3L(1, 128, 1);
    }
    if (max_mt == 2) {
      if (alt) TC3L(2, 128, 1);
      TC3L(2, 64, 1);
    }
    if (alt) TC3L(4, 64, 2);
    TC3L(4, 64, 1);
  }
  if (max_mt == 1) {
    if (alt) TC3L(1, 128, 2);
    TC3L(1, 128, 3);
  }
  if (max_mt == 2) {
    if (alt) TC3L(2, 64, 2);
    TC3L(2, 128, 2);
  }
  if (alt) TC3L(4, 64, 1);
  TC3L(4, 64, 2);
#undef TC3L
}


// ================================================================== V^ stage with swapped operand roles
// The low-rank V^ stage, mid_p = V^ t_src(p), applied to up to 128 pairs: the gathered source coefficient
// vectors are the A operand (M = 128 rows = pair x right-hand-side columns, K-major, the same 16-byte
// cp.async gathers as above) and the rows of V^'s real expansion are the B operand (N = 2r rounded up to 16,
// taken from the same pre-expanded operator image by cp.async.bulk). The accumulator is 128 TMEM lanes x
// NB columns, so a rank of 16 needs 32 columns instead of 128 lanes x 128 columns in the other orientation:
// up to 8 CTAs fit on an SM. Epilogue: lane = pair, so each thread writes its pair's 2r outputs as
// consecutive 16-byte stores into the low-rank intermediate.
template <int NB, int NST, int KCW = TC3_KC>
struct VswSmem {
  alignas(1024) float a[NST][128 * KCW];  // gathered coefficient vectors (128 rows x KCW real K)
  alignas(1024) float b[NST][NB * KCW];   // operator rows (NB rows x KCW real K)
  alignas(8) uint64_t bfull[NST];
  uint64_t mdone[NST];
  uint32_t tmem;
  int64_t sbase[128], dbase[128];
  int srr[128];
};

#define VSW_NT 128

// KCW: real K per pipeline chunk, 32 (one image chunk) or 16 (half of one: two chunks in flight in the shared
// memory one 32-wide chunk takes, so a chunk's gathers overlap the previous chunk's MMAs at the same CTAs per SM)
template <int NB, int NST, int KCW>
static __global__ void __launch_bounds__(VSW_NT, 8) k_m2l_vsw(const GemmUnit* units, const float* img,
                                                          const int64_t* psrc, const int64_t* pmid,
                                                          const float2* cout, float2* mid, int nrhs, int64_t ldc,
                                                          int64_t ldm, int* err) {
  typedef VswSmem<NB, NST, KCW> Sm;
  constexpr int HALVES = TC3_KC / KCW;      // pipeline chunks per image chunk (1 or 2)
  constexpr uint32_t SBO = (KCW / 4) * 128; // bytes between 8-row core-matrix groups
  extern __shared__ unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int D = NST - 1;
  const GemmUnit U = units[blockIdx.x];  // mode 1: M = r rows of V^, K = s
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int MT = (2 * U.M + 127) / 128;  // operator image tiles (1 or 2)
  const int nmma = ((2 * U.M + 15) / 16) * 16;
  const int nki = (2 * U.K + TC3_KC - 1) / TC3_KC;  // image chunks
  const int nk = (2 * U.K + KCW - 1) / KCW;          // pipeline chunks
  const float* A = img + U.a_off;
  const uint32_t idesc = idesc_tf32(128, nmma);
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(NB));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&S.bfull[q], 1);
      mbar_init(&S.mdone[q], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;
  uint32_t ph_b[NST], ph_m[NST];
#pragma unroll
  for (int q = 0; q < NST; ++q) ph_b[q] = ph_m[q] = 0;
  bool ok = true;
  auto wait_mdone = [&](int q) {
    bool mine = mbar_wait(&S.mdone[q], ph_m[q]);
    bool all = __syncthreads_and(mine ? 1 : 0) != 0;
    if (!all) {
      if (t == 0) atomicExch(err, 1);
      mbar_wait(&S.mdone[q], ph_m[q]);  // second bounded wait for MMAs still in flight
    }
    ph_m[q] ^= 1;
    return all;
  };
  auto issue = [&](int kc) {
    const int q = kc % NST;
    const int ic = kc / HALVES, h = kc % HALVES;  // image chunk and half
    if (HALVES == 1) {
      if (t == 0) {
        uint32_t bytes = 0;
        for (int mt = 0; mt < MT; ++mt) bytes += (uint32_t)tc3_ng(U.M, mt) * 1024u;
        tc3_expect_tx(&S.bfull[q], bytes);
        for (int mt = 0; mt < MT; ++mt) {
          const int ng = tc3_ng(U.M, mt);
          tc3_bulk(S.b[q] + mt * 16 * 256, A + (int64_t)16 * mt * nki * 256 + (int64_t)ic * ng * 256,
                   (uint32_t)ng * 1024u, &S.bfull[q]);
        }
      }
    } else {
      // half of every 8-row group (the group's first or last four K core matrices, 512 contiguous bytes)
      if (w == 0) {
        const int ng0 = tc3_ng(U.M, 0), ngt = ng0 + (MT > 1 ? tc3_ng(U.M, 1) : 0);
        if (lane == 0) tc3_expect_tx(&S.bfull[q], (uint32_t)ngt * 512u);
        __syncwarp();
        for (int gi = lane; gi < ngt; gi += 32) {
          const int mt = gi < ng0 ? 0 : 1, g = gi < ng0 ? gi : gi - ng0, ng = tc3_ng(U.M, mt);
          tc3_bulk(S.b[q] + (mt * 16 + g) * (8 * KCW),
                   A + (int64_t)16 * mt * nki * 256 + (int64_t)ic * ng * 256 + (int64_t)g * 256 + h * (8 * KCW),
                   512u, &S.bfull[q]);
        }
      }
    }
    const uint32_t abase = smem_u32(S.a[q]);
    // 16-byte segments (two complex values): KCW / 4 per row, consecutive threads along a row
    for (int seg = t; seg < 128 * (KCW / 4); seg += VSW_NT) {
      const int n = seg / (KCW / 4), j = seg % (KCW / 4);
      if (S.sbase[n] < 0) continue;  // unused row: its results are never read
      const int gj = kc * (KCW / 2) + 2 * j;
      const uint32_t dst = abase + kmaj_off(n, 4 * j, KCW);
      const float2* src = gj < U.K ? cout + (int64_t)S.srr[n] * ldc + S.sbase[n] + gj : cout;
      const uint32_t nbytes = gj + 1 < U.K ? 16u : (gj < U.K ? 8u : 0u);  // the rest is zero-filled
      if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        tc3_cp16(dst, src, nbytes);
      } else {
        tc3_cp8(dst, src, nbytes >= 8 ? 8u : 0u);
        tc3_cp8(dst + 8, nbytes == 16 ? src + 1 : cout, nbytes == 16 ? 8u : 0u);
      }
    }
    tc3_commit_group();
  };

  const int ncols = U.p_count * nrhs;
  for (int c0 = 0; c0 < ncols && ok; c0 += 128) {
    {
      const int c = c0 + t;
      if (c < ncols) {
        const int p = c / nrhs, rr = c - p * nrhs;
        const int64_t pi = U.p_begin + p;
        S.sbase[t] = psrc[pi];
        S.dbase[t] = pmid[pi];
        S.srr[t] = rr;
      } else {
        S.sbase[t] = -1;
        S.dbase[t] = -1;
        S.srr[t] = 0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < D; ++j) {
      if (j < nk)
        issue(j);
      else
        tc3_commit_group();
    }
    for (int kc = 0; kc < nk; ++kc) {
      const int j = kc + D;
      if (j < nk) {
        if (j >= NST) ok = wait_mdone(j % NST) && ok;
        issue(j);
      } else {
        tc3_commit_group();
      }
      tc3_wait_group<D>();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (t == 0) {
        const int q = kc % NST;
        if (!mbar_wait(&S.bfull[q], ph_b[q])) atomicExch(err, 1);
        ph_b[q] ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int s8 = 0; s8 < KCW / 8; ++s8) {
          if (kc * KCW + s8 * 8 >= 2 * U.K) break;  // K steps past the operator hold only zeros
          const uint64_t ad = smem_desc(smem_u32(S.a[q]) + s8 * 256, 128, SBO);
          const uint64_t bd = smem_desc(smem_u32(S.b[q]) + s8 * 256, 128, SBO);
          tc_mma(tmem, ad, bd, idesc, (kc > 0 || s8 > 0) ? 1 : 0);
        }
        tc_commit(&S.mdone[q]);
      }
    }
    for (int c = max(0, nk - NST); c < nk; ++c) ok = wait_mdone(c % NST) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int n = 32 * w + lane;  // TMEM lane = pair column
      const int64_t db = S.dbase[n];
      float* dst = db >= 0 ? reinterpret_cast<float*>(mid + (int64_t)S.srr[n] * ldm + db) : nullptr;
      const int nout = ((2 * U.M + 3) / 4) * 4;  // real outputs, rounded up to whole 16-byte stores (even-padded)
#pragma unroll 1
      for (int col0 = 0; col0 < nmma; col0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)col0, v);
        if (dst) {
#pragma unroll
          for (int q = 0; q < 32; q += 4)
            if (col0 + q < nout)
              *reinterpret_cast<float4*>(dst + col0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NB));
  }
}

template <int NB, int NST, int KCW>
static int vsw_launch_t(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc,
                        const int64_t* pmid, const float2* cout, float2* mid, int nrhs, int64_t ldc, int64_t ldm,
                        int* err, cudaStream_t s) {
  const size_t smem = sizeof(VswSmem<NB, NST, KCW>) + 1024;
  static bool attr = false;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_m2l_vsw<NB, NST, KCW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  for (size_t u0 = 0; u0 < nunits; u0 += 65535) {
    unsigned n = (unsigned)std::min<size_t>(65535, nunits - u0);
    k_m2l_vsw<NB, NST, KCW><<<n, VSW_NT, smem, s>>>(units + u0, img, psrc, pmid, cout, mid, nrhs, ldc, ldm, err);
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// The swapped V^ kernel for units whose rank r satisfies round16(2 r) <= nb (nb = 32, 64, 128 or 256 TMEM
// columns); nst = 1 or 2 pipeline stages of 32-wide chunks, or -2 / -3 for two / three stages of 16-wide ones.
int m2l_vsw_launch(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc, const int64_t* pmid,
                   const float2* cout, float2* mid, int nrhs, int64_t ldc, int64_t ldm, int nb, int nst, int* err,
                   cudaStream_t s) {
  if (nunits == 0) return FDA_OK;
#define VSWL(B_, S_, W_) \
  return vsw_launch_t<B_, S_, W_>(units, nunits, img, psrc, pmid, cout, mid, nrhs, ldc, ldm, err, s)
  if (nst == 1) {
    if (nb == 32) VSWL(32, 1, 32);
    if (nb == 64) VSWL(64, 1, 32);
    if (nb == 128) VSWL(128, 1, 32);
    if (nb == 256) VSWL(256, 1, 32);
  } else if (nst == 2) {
    if (nb == 32) VSWL(32, 2, 32);
    if (nb == 64) VSWL(64, 2, 32);
    if (nb == 128) VSWL(128, 2, 32);
    if (nb == 256) VSWL(256, 2, 32);
  } else if (nst == -2) {  // 16-wide chunks, two in flight
    if (nb == 32) VSWL(32, 2, 16);
    if (nb == 64) VSWL(64, 2, 16);
    if (nb == 128) VSWL(128, 2, 16);
    if (nb == 256) VSWL(256, 2, 16);
  } else if (nst == -3) {  // 16-wide chunks, three in flight
    if (nb == 32) VSWL(32, 3, 16);
    if (nb == 64) VSWL(64, 3, 16);
    if (nb == 128) VSWL(128, 3, 16);
    if (nb == 256) VSWL(256, 3, 16);
  }
#undef VSWL
  set_error("swapped V^ kernel: no variant for %d TMEM columns and %d stages", nb, nst);
  return FDA_E_INVALID_ARG;
}


// ================================================================== V^ stage fed by TMA row gathers
// The swapped V^ kernel for one right-hand side with its gathered A operand loaded by the tensor memory
// accelerator: the level's coefficient vectors are a 2-D tensor (rows of 2 s floats), and a K chunk of 128
// rows x 32 floats is 32 cp.async.bulk.tensor tile::gather4 loads (four rows each, one per lane of warp 0)
// into the 128-byte-swizzled K-major layout the MMA reads (8-row atoms of 1 KB). The operator rows come by
// cp.async.bulk as before; both complete on the stage's mbarrier. Warp 0 runs the pipeline: lookahead
// NST - 1 chunks, lane 0 issues the MMAs and commits each stage; the four warps share the epilogue.
template <int NB, int NST>
struct VtmSmem {
  alignas(1024) float a[NST][128 * TC3_KC];  // gathered rows, 128-byte swizzle
  alignas(1024) float b[NST][NB * TC3_KC];   // operator rows, canonical layout without swizzle
  alignas(8) uint64_t full[NST];
  uint64_t mdone[NST];
  uint32_t tmem;
  int rows[128];
  int64_t dbase[128];
};

// shared-memory descriptor of a K-major operand in the 128-byte swizzle (8-row atoms of 1 KB)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset: one 8-row atom
  d |= (uint64_t)1 << 46;               // version
  d |= (uint64_t)2 << 61;               // layout: 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, int x, int y0, int y1, int y2,
                                            int y3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_u32(bar))
      : "memory");
}

template <int NB, int NST>
static __global__ void __launch_bounds__(VSW_NT) k_m2l_vtm(const GemmUnit* units, const float* img,
                                                          const int64_t* psrc, const int64_t* pmid, float2* mid,
                                                          int64_t base, int s_l, int* err,
                                                          const __grid_constant__ CUtensorMap tmap) {
  typedef VtmSmem<NB, NST> Sm;
  extern __shared__ unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int D = NST - 1;
  const GemmUnit U = units[blockIdx.x];  // mode 1: M = r rows of V^, K = s
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int MT = (2 * U.M + 127) / 128;
  const int nmma = ((2 * U.M + 15) / 16) * 16;
  const int nk = (2 * U.K + TC3_KC - 1) / TC3_KC;
  const float* A = img + U.a_off;
  const uint32_t idesc = idesc_tf32(128, nmma);
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(NB));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&S.full[q], 1);
      mbar_init(&S.mdone[q], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  {
    // rows past the unit's pairs repeat its first source (their results are not stored)
    const int p = t < U.p_count ? t : 0;
    S.rows[t] = (int)((psrc[U.p_begin + p] - base) / s_l);
    S.dbase[t] = t < U.p_count ? pmid[U.p_begin + t] : -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;
  int ok = 1;
  if (w == 0) {
    const int y0 = S.rows[4 * lane], y1 = S.rows[4 * lane + 1], y2 = S.rows[4 * lane + 2], y3 = S.rows[4 * lane + 3];
    for (int step = 0; step < nk + D && ok; ++step) {
      if (step < nk) {  // load chunk `step`
        const int q = step % NST;
        if (step >= NST) {
          int mine = lane == 0 ? (mbar_wait(&S.mdone[q], (uint32_t)((step / NST - 1) & 1)) ? 1 : 0) : 1;
          ok = __shfl_sync(0xffffffffu, mine, 0);
          if (!ok) break;
        }
        if (lane == 0) {
          uint32_t bytes = 128u * TC3_KC * 4u;
          for (int mt = 0; mt < MT; ++mt) bytes += (uint32_t)tc3_ng(U.M, mt) * 1024u;
          tc3_expect_tx(&S.full[q], bytes);
          for (int mt = 0; mt < MT; ++mt) {
            const int ng = tc3_ng(U.M, mt);
            tc3_bulk(S.b[q] + mt * 16 * 256, A + (int64_t)16 * mt * nk * 256 + (int64_t)step * ng * 256,
                     (uint32_t)ng * 1024u, &S.full[q]);
          }
        }
        __syncwarp();
        tma_gather4(smem_u32(S.a[q]) + 512u * (uint32_t)lane, &tmap, TC3_KC * step, y0, y1, y2, y3, &S.full[q]);
      }
      const int kc = step - D;
      if (kc >= 0) {  // MMAs of chunk kc
        const int q = kc % NST;
        int mine = 1;
        if (lane == 0) {
          if (!mbar_wait(&S.full[q], (uint32_t)((kc / NST) & 1))) {
            mine = 0;
          } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s8 = 0; s8 < TC3_KC / 8; ++s8) {
              if (kc * TC3_KC + s8 * 8 >= 2 * U.K) break;
              const uint64_t ad = smem_desc_sw128(smem_u32(S.a[q]) + 32u * (uint32_t)s8);
              const uint64_t bd = smem_desc(smem_u32(S.b[q]) + s8 * 256, 128, (TC3_KC / 4) * 128);
              tc_mma(tmem, ad, bd, idesc, (kc > 0 || s8 > 0) ? 1 : 0);
            }
            tc_commit(&S.mdone[q]);
          }
        }
        ok = __shfl_sync(0xffffffffu, mine, 0);
      }
    }
  }
  // the last chunk's commit covers every MMA of the unit
  const int qlast = (nk - 1) % NST;
  bool mine = mbar_wait(&S.mdone[qlast], (uint32_t)(((nk - 1) / NST) & 1));
  const bool all = __syncthreads_and((mine && (w != 0 || ok)) ? 1 : 0) != 0;
  if (!all && t == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (all) {
    const int n = 32 * w + lane;  // TMEM lane = pair
    const int64_t db = S.dbase[n];
    float* dst = db >= 0 ? reinterpret_cast<float*>(mid + db) : nullptr;
    const int nout = ((2 * U.M + 3) / 4) * 4;
#pragma unroll 1
    for (int col0 = 0; col0 < nmma; col0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)col0, v);
      if (dst) {
#pragma unroll
        for (int q = 0; q < 32; q += 4)
          if (col0 + q < nout) *reinterpret_cast<float4*>(dst + col0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  } else {
    // a wait gave up: let every copy issued into this CTA's buffers land (bounded) before it leaves
    for (int q = 0; q < NST; ++q) mbar_wait(&S.full[q], 0u), mbar_wait(&S.full[q], 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NB));
  }
}

template <int NB, int NST>
static int vtm_launch_t(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc,
                        const int64_t* pmid, float2* mid, int64_t base, int s_l, const CUtensorMap* map, int* err,
                        cudaStream_t s) {
  const size_t smem = sizeof(VtmSmem<NB, NST>) + 1024;
  static bool attr = false;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_m2l_vtm<NB, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  for (size_t u0 = 0; u0 < nunits; u0 += 65535) {
    unsigned n = (unsigned)std::min<size_t>(65535, nunits - u0);
    k_m2l_vtm<NB, NST><<<n, VSW_NT, smem, s>>>(units + u0, img, psrc, pmid, mid, base, s_l, err, *map);
    FDA_LAUNCH_CHECK();
  }
  return FDA_OK;
}

// one right-hand side; nb = 32, 64, 128 or 256 TMEM columns (round16(2 r) <= nb), nst = 2, 3 or 4 stages
int m2l_vtm_launch(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc, const int64_t* pmid,
                   float2* mid, int64_t base, int s_l, const CUtensorMap* map, int nb, int nst, int* err,
                   cudaStream_t s) {
  if (nunits == 0) return FDA_OK;
#define VTML(B_, S_) return vtm_launch_t<B_, S_>(units, nunits, img, psrc, pmid, mid, base, s_l, map, err, s)
  if (nst == 2) {
    if (nb == 32) VTML(32, 2);
    if (nb == 64) VTML(64, 2);
    if (nb == 128) VTML(128, 2);
    if (nb == 256) VTML(256, 2);
  } else if (nst == 3) {
    if (nb == 32) VTML(32, 3);
    if (nb == 64) VTML(64, 3);
    if (nb == 128) VTML(128, 3);
    if (nb == 256) VTML(256, 3);
  } else {
    if (nb == 32) VTML(32, 4);
    if (nb == 64) VTML(64, 4);
    if (nb == 128) VTML(128, 4);
  }
#undef VTML
  set_error("TMA-fed V^ kernel: no variant for %d TMEM columns and %d stages", nb, nst);
  return FDA_E_INVALID_ARG;
}

// ================================================================== persistent, warp-specialised scatter stage
// For units whose K fits two 32-wide real chunks (the U^ stage of low-rank pairs, mode 2, and dense units
// with K <= 32 complex, mode 0) the operator of a unit is loaded once and stays in shared memory while the
// unit's columns stream through in blocks of WS_NB:
//  - warps 0-2 (producers): 16-byte cp.async gathers of a block's source vectors into a ring of WS_NS
//    stages, each thread signalling the stage's "full" mbarrier with cp.async.mbarrier.arrive.noinc; thread
//    0 also loads each unit's operator tiles (cp.async.bulk, transaction bytes on an mbarrier);
//  - warp 3, lane 0 (MMA): tcgen05.mma of all row tiles into one of two TMEM accumulators, committing the
//    ring stage, the accumulator and, after a unit's last block, the operator buffer;
//  - warps 4-7 (epilogue, TMEM lane quadrant w - 4): accumulators through shared memory, one
//    cp.reduce.async.bulk per column into the target vectors, then the accumulator is handed back.
// CTAs are persistent (one per SM) and take units round-robin. Every wait is bounded; a wait that gives up
// sets the CTA's abort flag (and the error flag), every role leaves its loop at its next check, and the
// epilogue warps decide together through a shared slot so that their named barrier never splits.
#define WS_NB 32   // columns per block
#define WS_NS 3    // ring stages
#define WS_NT 256

template <int MTC>
struct WsSmem {
  alignas(1024) float a[MTC][2][128 * TC3_KC];         // operator tiles, two K chunks
  alignas(1024) float b[WS_NS][2][WS_NB * TC3_KC];     // gathered columns
  alignas(1024) float stg[2][16 * 128 * MTC];          // epilogue staging: 16 columns x real rows
  alignas(8) uint64_t a_full, a_empty;
  uint64_t b_full[WS_NS], b_empty[WS_NS];
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem;
  int abort_flag, epi_fail, epi_abort;
};

__device__ __forceinline__ void ws_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void ws_cp_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void ws_epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int MTC>
static __global__ void __launch_bounds__(WS_NT, 1) k_m2l_ws(const GemmUnit* units, int nunits, const float* img,
                                                           const int64_t* psrc, const int64_t* ptgt,
                                                           const int64_t* pmid, const float2* cout, float2* cin,
                                                           const float2* mid, int nrhs, int64_t ldc, int64_t ldm,
                                                           int* err) {
  typedef WsSmem<MTC> Sm;
  extern __shared__ unsigned char smem_raw[];
  Sm& S = *reinterpret_cast<Sm*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int TCOLS = 2 * MTC * WS_NB <= 256 ? 256 : 512;
  constexpr uint32_t IDESC = idesc_tf32(128, WS_NB);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    mbar_init(&S.a_full, 1);
    mbar_init(&S.a_empty, 1);
    for (int q = 0; q < WS_NS; ++q) {
      mbar_init(&S.b_full[q], 96);  // one cp.async arrival per producer thread
      mbar_init(&S.b_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&S.acc_full[q], 1);
      mbar_init(&S.acc_empty[q], 4);  // lane 0 of each epilogue warp
    }
    S.abort_flag = 0;
    S.epi_fail = 0;
    S.epi_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;
  volatile int* abort_flag = &S.abort_flag;
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicExch(err, 1);
  };

  if (w < 3) {
    // ------------------------------------------------------------ producers
    int64_t g = 0;  // block counter over this CTA's units
    int ui = 0, a_loads = 0;
    for (int u = blockIdx.x; u < nunits && !*abort_flag; u += gridDim.x, ++ui) {
      const GemmUnit U = units[u];
      const float2* X = U.mode == 2 ? mid : cout;
      const int64_t lds = U.mode == 2 ? ldm : ldc;
      const int MT = (2 * U.M + 127) / 128, nk = (2 * U.K + TC3_KC - 1) / TC3_KC;
      if (t == 0) {
        if (ui > 0 && !mbar_wait(&S.a_empty, (ui - 1) & 1)) give_up();
        if (!*abort_flag) {
          uint32_t bytes = 0;
          for (int mt = 0; mt < MT; ++mt) bytes += (uint32_t)nk * tc3_ng(U.M, mt) * 1024u;
          tc3_expect_tx(&S.a_full, bytes);
          ++a_loads;
          const float* A = img + U.a_off;
          for (int mt = 0; mt < MT; ++mt) {
            const int ng = tc3_ng(U.M, mt);
            for (int kc = 0; kc < nk; ++kc)
              tc3_bulk(S.a[mt][kc], A + (int64_t)16 * mt * nk * 256 + (int64_t)kc * ng * 256, (uint32_t)ng * 1024u,
                       &S.a_full);
          }
        }
      }
      const int ncols = U.p_count * nrhs;
      for (int c0 = 0; c0 < ncols && !*abort_flag; c0 += WS_NB, ++g) {
        const int st = (int)(g % WS_NS);
        if (g >= WS_NS && !mbar_wait(&S.b_empty[st], (uint32_t)((g / WS_NS - 1) & 1))) {
          give_up();
          break;
        }
        // WS_NB columns x nk chunks x 8 segments of 16 bytes; 8 consecutive threads read one column's chunk
        for (int seg = t; seg < WS_NB * 16; seg += 96) {
          const int j = seg & 7, kc = (seg >> 3) & 1, n = seg >> 4;
          if (kc >= nk) continue;
          const int c = c0 + n;
          if (c >= ncols) continue;
          const int p = c / nrhs, rr = c - p * nrhs;
          const int64_t pi = U.p_begin + p;
          const int64_t sb = U.mode == 2 ? pmid[pi] : psrc[pi];
          const int gj = kc * (TC3_KC / 2) + 2 * j;
          const uint32_t dst = smem_u32(S.b[st][kc]) + kmaj_off(n, 4 * j, TC3_KC);
          const float2* src = gj < U.K ? X + (int64_t)rr * lds + sb + gj : X;
          const uint32_t nbytes = gj + 1 < U.K ? 16u : (gj < U.K ? 8u : 0u);
          if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            tc3_cp16(dst, src, nbytes);
          } else {
            tc3_cp8(dst, src, nbytes >= 8 ? 8u : 0u);
            tc3_cp8(dst + 8, nbytes == 16 ? src + 1 : X, nbytes == 16 ? 8u : 0u);
          }
        }
        ws_cp_arrive(&S.b_full[st]);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the last operator load has landed before the CTA can leave (it already has unless the CTA aborted)
    if (t == 0 && a_loads > 0) mbar_wait(&S.a_full, (uint32_t)((a_loads - 1) & 1));
  } else if (w == 3) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int64_t g = 0;
      int ui = 0;
      bool pending = false;  // an accumulator commit whose MMAs may still run
      uint32_t last_buf = 0, last_par = 0;
      for (int u = blockIdx.x; u < nunits && !*abort_flag; u += gridDim.x, ++ui) {
        const GemmUnit U = units[u];
        const int MT = (2 * U.M + 127) / 128, nk = (2 * U.K + TC3_KC - 1) / TC3_KC;
        if (!mbar_wait(&S.a_full, ui & 1)) {
          give_up();
          break;
        }
        const int ncols = U.p_count * nrhs;
        for (int c0 = 0; c0 < ncols && !*abort_flag; c0 += WS_NB, ++g) {
          const int st = (int)(g % WS_NS);
          const uint32_t buf = (uint32_t)(g & 1);
          if (g >= 2 && !mbar_wait(&S.acc_empty[buf], (uint32_t)(((g >> 1) - 1) & 1))) {
            give_up();
            break;
          }
          if (!mbar_wait(&S.b_full[st], (uint32_t)((g / WS_NS) & 1))) {
            give_up();
            break;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // gathered data -> async proxy
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d0 = tmem + buf * (uint32_t)(MTC * WS_NB);
          for (int mt = 0; mt < MT; ++mt)
            for (int kc = 0; kc < nk; ++kc)
#pragma unroll
              for (int s8 = 0; s8 < TC3_KC / 8; ++s8) {
                if (kc * TC3_KC + s8 * 8 >= 2 * U.K) break;
                const uint64_t ad = smem_desc(smem_u32(S.a[mt][kc]) + s8 * 256, 128, (TC3_KC / 4) * 128);
                const uint64_t bd = smem_desc(smem_u32(S.b[st][kc]) + s8 * 256, 128, (TC3_KC / 4) * 128);
                tc_mma(d0 + (uint32_t)(WS_NB * mt), ad, bd, IDESC, (kc > 0 || s8 > 0) ? 1 : 0);
              }
          tc_commit(&S.b_empty[st]);
          tc_commit(&S.acc_full[buf]);
          pending = true;
          last_buf = buf;
          last_par = (uint32_t)((g >> 1) & 1);
          if (c0 + WS_NB >= ncols) tc_commit(&S.a_empty);
        }
      }
      // on an abort, the MMAs already issued finish before the accumulators are released
      if (*abort_flag && pending) mbar_wait(&S.acc_full[last_buf], last_par);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q4 = w - 4;
    int64_t g = 0;
    int grp = 0;  // staging group counter
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
      const GemmUnit U = units[u];
      const int MT = (2 * U.M + 127) / 128;
      const int RT = 128 * MT;
      const int ncols = U.p_count * nrhs;
      bool stop = false;
      for (int c0 = 0; c0 < ncols; c0 += WS_NB, ++g) {
        const uint32_t buf = (uint32_t)(g & 1);
        // one decision for the four epilogue warps: any abort, or any of their waits giving up
        const bool mine = mbar_wait(&S.acc_full[buf], (uint32_t)((g >> 1) & 1));
        if (!mine) atomicOr(&S.epi_fail, 1);
        ws_epi_sync();
        if (t == 128) S.epi_abort = (S.epi_fail || *abort_flag) ? 1 : 0;
        ws_epi_sync();
        if (S.epi_abort) {
          if (t == 128) give_up();
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d0 = tmem + buf * (uint32_t)(MTC * WS_NB);
        for (int cg = 0; cg < WS_NB / 16; ++cg, ++grp) {
          float* sb = S.stg[grp & 1];
          if (t >= 128 && t < 144) bulk_wait_read<1>();
          ws_epi_sync();
          for (int mt = 0; mt < MT; ++mt) {
            float v[16];
            tmem_ld16(d0 + ((uint32_t)(32 * q4) << 16) + (uint32_t)(WS_NB * mt + 16 * cg), v);
            const int row = 128 * mt + 32 * q4 + lane;
#pragma unroll
            for (int c = 0; c < 16; ++c) sb[c * RT + row] = v[c];
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          ws_epi_sync();
          if (t >= 128 && t < 144) {
            const int c = c0 + 16 * cg + (t - 128);
            if (c < ncols) {
              const int p = c / nrhs, rr = c - p * nrhs;
              float2* dst = cin + (int64_t)rr * ldc + ptgt[U.p_begin + p];
              if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (U.M & 1) == 0)
                bulk_reduce_add(dst, sb + (t - 128) * RT, 8u * (uint32_t)U.M);
              else
                atomicExch(err, 2);  // never made by a plan: reported, skipped
            }
            bulk_commit();
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) ws_arrive(&S.acc_empty[buf]);
      }
      if (stop) break;
    }
    if (t >= 128 && t < 144) bulk_wait_read<0>();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

template <int MTC>
static int ws_launch_t(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc,
                       const int64_t* ptgt, const int64_t* pmid, const float2* cout, float2* cin, const float2* mid,
                       int nrhs, int64_t ldc, int64_t ldm, int* err, cudaStream_t s) {
  const size_t smem = sizeof(WsSmem<MTC>) + 1024;
  static bool attr = false;
  static int nsm = 0;
  if (!attr) {
    FDA_CUDA(cudaFuncSetAttribute(k_m2l_ws<MTC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0;
    FDA_CUDA(cudaGetDevice(&dev));
    FDA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    attr = true;
  }
  const unsigned grid = (unsigned)std::min<size_t>(nunits, (size_t)std::max(1, nsm));
  k_m2l_ws<MTC><<<grid, WS_NT, smem, s>>>(units, (int)nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm,
                                          err);
  FDA_LAUNCH_CHECK();
  return FDA_OK;
}

// units: modes 0 or 2 with 2 K <= 64 real columns, even M; max_mt: largest row-tile count (<= 4)
int m2l_ws_launch(const GemmUnit* units, size_t nunits, const float* img, const int64_t* psrc, const int64_t* ptgt,
                  const int64_t* pmid, const float2* cout, float2* cin, const float2* mid, int nrhs, int64_t ldc,
                  int64_t ldm, int max_mt, int* err, cudaStream_t s) {
  if (nunits == 0) return FDA_OK;
  if (nunits > (size_t)INT32_MAX) {
    set_error("too many units for the persistent scatter kernel");
    return FDA_E_INVALID_ARG;
  }
  if (max_mt <= 2) return ws_launch_t<2>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s);
  if (max_mt == 3) return ws_launch_t<3>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s);
  if (max_mt == 4) return ws_launch_t<4>(units, nunits, img, psrc, ptgt, pmid, cout, cin, mid, nrhs, ldc, ldm, err, s);
  set_error("persistent scatter kernel: at most 4 row tiles (got %d)", max_mt);
  return FDA_E_INVALID_ARG;
}

}  // namespace fda

using namespace fda;

// Failure-detection self-test: one thread waits on an mbarrier phase that nothing completes, with the given
// wall-clock bound; when the bound runs out it records the timeout and returns (no trap, no fault).
static __global__ void k_wait_probe(uint64_t limit_ns, int* timed_out) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t a = smem_u32(&bar);
    const uint64_t t0 = tc_clock_ns();
    int done = 0;
    while (!done) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(a), "r"(0u)
          : "memory");
      if (ok) done = 1;
      else if (tc_clock_ns() - t0 > limit_ns) done = 2;
    }
    *timed_out = done == 2 ? 1 : 0;
  }
}

// Self-test of the tensor-core path: one complex M x K product applied to P gathered columns, against an FP64
// host product of the same FP32 data. split 0: TF32 (M = 64, P = 64); 1: 3xTF32 split (M = 64, P = 64);
// 2..7: TF32 with the pre-expanded operator image (M = min(256, K), P = 100), tile shape split - 2 (6 and 7:
// the bulk-reduction epilogue); 8, 9: the swapped-operand V^ kernel with one or two stages (M = min(100, K),
// P = 100, results stored into an intermediate with even-padded vectors as the low-rank stage does);
// 10, 11: 3xTF32 from the TF32 and remainder images (atomics, bulk reductions); 12, 13: the swapped V^ kernel
// with 16-wide K chunks (two and three in flight).
extern "C" int fda_tc_selftest(int K, int split, double* max_rel_err, int* wait_failed) {
  if (K < 1 || K > 1024 || split < 0 || split > 13 || !max_rel_err || !wait_failed) {
    set_error("bad arguments");
    return FDA_E_INVALID_ARG;
  }
  const bool vsw = split == 8 || split == 9 || split == 12 || split == 13;
  const bool x3 = split == 10 || split == 11;
  // the bulk-reduction epilogue adds whole 16-byte granules: even row counts (as every plan has)
  const bool bulk = split == 6 || split == 7 || split == 11;
  const int Mb = bulk ? std::min(256, (K + 1) & ~1) : std::min(256, K);
  const int M = vsw ? std::min(100, K) : (split >= 2 ? Mb : 64), P = split >= 2 ? 100 : 64;
  const int Mp = vsw ? (M + 1) & ~1 : M;  // stride of the stored vectors
  std::vector<float2> hA((size_t)M * K), hX((size_t)K * P);
  uint64_t st = 12345;
  auto rnd = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((double)(st >> 11) / 9007199254740992.0 * 2.0 - 1.0);
  };
  for (auto& a : hA) a = make_float2(rnd(), rnd());
  for (auto& x : hX) x = make_float2(rnd(), rnd());
  DBuf<float2> dA, dX, dY, dmid;
  DBuf<int64_t> src, tgt, pm;
  DBuf<GemmUnit> du;
  DBuf<int> err;
  std::vector<int64_t> hs(P), ht(P), hm(P, -1);
  for (int p = 0; p < P; ++p) hs[p] = (int64_t)p * K, ht[p] = (int64_t)p * M, hm[p] = vsw ? (int64_t)p * Mp : -1;
  FDA_TRY(dA.upload(hA));
  FDA_TRY(dX.upload(hX));
  FDA_TRY(dY.alloc((size_t)Mp * P));
  FDA_TRY(dY.zero());
  FDA_TRY(dmid.alloc(vsw ? (size_t)P * Mp : 1));
  FDA_TRY(dmid.zero());
  FDA_TRY(src.upload(hs));
  FDA_TRY(tgt.upload(ht));
  FDA_TRY(pm.upload(hm));
  FDA_TRY(err.alloc(1));
  FDA_TRY(err.zero());
  if (split >= 2) {
    std::vector<double2> hA64(hA.size());
    for (size_t q = 0; q < hA.size(); ++q) hA64[q] = make_double2(hA[q].x, hA[q].y);
    DBuf<double2> dA64;
    DBuf<float> img;
    FDA_TRY(dA64.upload(hA64));
    FDA_TRY(img.alloc((size_t)tc3_image_floats(M, K) * (x3 ? 2 : 1)));
    FDA_TRY(tc3_build_images({TcImgJob{dA64.p, M, K, 0, M, 0, x3 ? 1 : 0}}, img.p));
    GemmUnit u{0, M, K, 0, P, 0, vsw ? 1 : 0, 0};
    FDA_TRY(du.upload(&u, 1));
    if (vsw) {
      const int nm = ((2 * M + 15) / 16) * 16;
      const int nb = nm <= 32 ? 32 : nm <= 64 ? 64 : nm <= 128 ? 128 : 256;
      const int vst = split == 8 ? 1 : (split == 9 ? 2 : (split == 12 ? -2 : -3));
      FDA_TRY(m2l_vsw_launch(du.p, 1, img.p, src.p, pm.p, dX.p, dmid.p, 1, 0, 0, nb, vst, err.p, 0));
      FDA_CUDA(cudaDeviceSynchronize());
      FDA_CUDA(cudaMemcpy(dY.p, dmid.p, sizeof(float2) * P * Mp, cudaMemcpyDeviceToDevice));
    } else {
      FDA_TRY(m2l_tc3_launch(du.p, 1, img.p, src.p, tgt.p, pm.p, dX.p, dY.p, dmid.p, 1, 0, 0, (2 * M + 127) / 128,
                             K, err.p, 0, x3 ? split - 4 : split - 2));
    }
    FDA_CUDA(cudaDeviceSynchronize());
  } else {
    GemmUnit u{0, M, K, 0, P, 0, 0, 0};
    FDA_TRY(du.upload(&u, 1));
    FDA_TRY(m2l_tc_launch(du.p, 1, dA.p, dA.p, src.p, tgt.p, pm.p, dX.p, dY.p, dmid.p, 1, 0, 0, split, M, err.p, 0));
    FDA_CUDA(cudaDeviceSynchronize());
  }
  std::vector<float2> hY;
  FDA_TRY(dY.download(hY));
  int he = 0;
  FDA_CUDA(cudaMemcpy(&he, err.p, sizeof(int), cudaMemcpyDeviceToHost));
  double worst = 0;
  for (int p = 0; p < P; ++p)
    for (int i = 0; i < M; ++i) {
      double rr = 0, ri = 0, nrm = 0;
      for (int k = 0; k < K; ++k) {
        float2 a = hA[i + (size_t)k * M], x = hX[(size_t)p * K + k];
        rr += (double)a.x * x.x - (double)a.y * x.y;
        ri += (double)a.x * x.y + (double)a.y * x.x;
        nrm += sqrt(((double)a.x * a.x + (double)a.y * a.y) * ((double)x.x * x.x + (double)x.y * x.y));
      }
      float2 y = hY[(size_t)p * Mp + i];
      double e = sqrt((y.x - rr) * (y.x - rr) + (y.y - ri) * (y.y - ri)) / nrm;
      worst = std::max(worst, e);
    }
  *max_rel_err = worst;
  *wait_failed = he;
  return FDA_OK;
}

extern "C" int fda_wait_selftest(double limit_ms, int* timed_out) {
  if (!(limit_ms > 0 && limit_ms <= 1000.0) || !timed_out) {
    set_error("limit_ms must lie in (0, 1000]");
    return FDA_E_INVALID_ARG;
  }
  DBuf<int> d;
  FDA_TRY(d.alloc(1));
  FDA_TRY(d.zero());
  k_wait_probe<<<1, 32>>>((uint64_t)(limit_ms * 1e6), d.p);
  FDA_LAUNCH_CHECK();
  FDA_CUDA(cudaDeviceSynchronize());
  FDA_CUDA(cudaMemcpy(timed_out, d.p, sizeof(int), cudaMemcpyDeviceToHost));
  return FDA_OK;
}
