// Split-TF32 tensor-core form of the FP32 body stage kernel (sm_103a, tcgen05).
//
// Same computation as stage_kernel for a Hermitian run with real H and N <= 16 (see stage_kernel.cuh),
// except that the commutator's product S = s H of every ADO runs on the tensor cores:
//   -i (H s - s H) = i S - i S^dagger   (s and H Hermitian, so H s = S^dagger),
// and the owner-lane form adds Q + Q^dagger with Q = i S - (decay / 2) s + row links.
//
// A CTA is 4 warps.  Each warp keeps the software pipeline of stage_kernel over its own chunks of
// A = floor(32 / N) ADOs; the 4 warps meet once per chunk round, when lane (a, i) of warp w has written
// row i of ADO a (real and imaginary parts, each split into TF32 high and low parts) into tensor-memory
// lane 32 w + lane of four 16-column operand blocks (tcgen05.st; the A operand of the MMA sits in
// tensor memory, so the shared memory holds only H).  One thread then issues, per 8-wide K step,
//   D[:, 0:16)  += Re_hi H_hi + Re_lo H_hi + Re_hi H_lo
//   D[:, 16:32) += Im_hi H_hi + Im_lo H_hi + Im_hi H_lo
// as tcgen05.mma kind::tf32 (M = 128, N = 16, K = 8, FP32 accumulators in tensor memory) and commits
// them to an mbarrier.  The tensor cores run while every warp gathers its linked neighbours and
// applies the links; each warp then reads its 32 lanes of D (its own rows) with tcgen05.ld.  The
// dropped lo * lo term and the TF32 width of the parts leave about 21 correct bits of S.
// The B operand (H) uses the no-swizzle K-major shared-memory layout: 8-row x 16-byte core matrices,
// the 4 core matrices of one 8-row group adjacent (leading byte offset 128 B between K-adjacent core
// matrices, stride byte offset 512 B between 8-row groups).  Tensor memory of a CTA: columns 0-31 D
// (real | imaginary part of S), 32-95 the A blocks Re_hi, Re_lo, Im_hi, Im_lo.
// Every wait on the mbarrier gives up after about a second of clock cycles: the thread sets *c.err,
// the CTA stops at the next round and frees its tensor memory; the host reports HEOM_E_TIMEOUT.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "stage_kernel.cuh"

namespace heom {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// the column count is an immediate so that the kernel's tensor-memory use is known at compile time
template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot_smem), "n"(NCOLS)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "n"(NCOLS) : "memory");
}
// D (tensor memory) = A B^T (+ D when acc != 0); A, B described by shared-memory descriptors
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// the mbarrier completes one arrival when every tcgen05 operation this thread issued before has finished
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred P1;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
      "selp.b32 %0, 1, 0, P1;\n"
      "}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// D (tensor memory) = A B^T (+ D when acc != 0); A in tensor memory (row m in lane m, K in columns),
// B described by a shared-memory descriptor
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// 32 lanes x 16 columns of 32-bit tensor memory from one lane per thread of the warp
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n" ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// 32 lanes x 32 columns of 32-bit tensor memory, one lane per thread of the warp, then wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&u)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr)
      : "memory");
}

// Shared-memory matrix descriptor of a no-swizzle K-major operand (tcgen05 format: start address >> 4
// in bits 0-13, leading byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, version 1 in
// 46-47; base offset 0, leading-offset mode 0, layout type 0 = no swizzle in 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15 and 16 = 0), N >> 3 in bits 17-22, M >> 4 in 24-28.
constexpr uint32_t tf32_idesc(int M, int Nn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Nn >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

#ifndef HEOM_TC_REC_CAP
#define HEOM_TC_REC_CAP 12  // link records per warp and batch (x2: Hermitian row-only slices)
#endif
#ifndef HEOM_TC_MIN_BLOCKS
#define HEOM_TC_MIN_BLOCKS 4  // CTAs per SM the register allocation must allow (128 registers)
#endif
constexpr int kTcRC = HEOM_TC_REC_CAP;
constexpr int kTcWarps = 4;                          // 128 rows of D, one TMEM lane quarter per warp
constexpr int kTcCols = 128;                         // tensor-memory columns of a CTA (96 used)
constexpr int kTcA = 32;                             // first column of the A blocks
constexpr int kTcK = 16;                             // N padded: the K and N extents of every MMA
constexpr long long kTcWaitCycles = 2000000000LL;    // about a second at the GB300 SM clock

// Byte offset of element (row m, column k) in a 16-wide K-major no-swizzle shared-memory operand.
__device__ __forceinline__ int tc_off(int m, int k) {
  return ((m >> 3) * 4 + (k >> 2)) * 128 + (m & 7) * 16 + (k & 3) * 4;
}

// CTA-shared part of the dynamic shared memory (the per-warp stage buffers follow).
struct TcSmem {
  static constexpr int b_tile = 16 * kTcK * 4;   // 16 rows x 16 TF32
  static constexpr int b0 = 0;                   // H_hi, H_lo
  static constexpr int mbar = b0 + 2 * b_tile;
  static constexpr int tslot = mbar + 8;         // tensor-memory address written by tcgen05.alloc
  static constexpr int total = (tslot + 4 + 127) & ~127;
};

template <int N>
__global__ void __launch_bounds__(kTcWarps * 32, HEOM_TC_MIN_BLOCKS) stage_tc_kernel(const __grid_constant__ StageArgs<float> a) {
  static_assert(N >= 1 && N <= kTcK, "the tensor-core form covers n_states <= 16");
  using S = StageShape<N, float, float, kTcRC>;
  using W = WarpSmem<N, float, float, kTcRC>;
  using C2 = float2;
  using R = LinkRec<float>;
  constexpr int A = S::A, EPO = S::EpOwn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StageCommon &c = a.c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *cta = smem_raw;
  unsigned char *wb = smem_raw + TcSmem::total + warp * W::total;
  C2 *ybuf = reinterpret_cast<C2 *>(wb + W::ybuf);
  C2 *gbuf = reinterpret_cast<C2 *>(wb + W::gbuf);
  const uint32_t b_base = smem_u32(cta + TcSmem::b0);
  const uint32_t mbar = smem_u32(cta + TcSmem::mbar);

  // B operand: H split into TF32 parts, B[n][k] = H[k][n]; zero padding beyond N
  for (int idx = threadIdx.x; idx < 16 * kTcK; idx += kTcWarps * 32) {
    const int n = idx / kTcK, k = idx - n * kTcK;
    const float h = (n < N && k < N) ? a.H[k * kMaxStates + n] : 0.f;
    const float hi = to_tf32(h), lo = to_tf32(h - hi);
    *reinterpret_cast<float *>(cta + TcSmem::b0 + tc_off(n, k)) = hi;
    *reinterpret_cast<float *>(cta + TcSmem::b0 + TcSmem::b_tile + tc_off(n, k)) = lo;
  }
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc<kTcCols>(smem_u32(cta + TcSmem::tslot));
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(cta + TcSmem::tslot);

  const int la = lane / N;
  const int li = lane - la * N;
  const bool lane_ok = la < A;
  const bool has_y = c.y.body != nullptr;
  const bool same_y = c.y.body == c.zin.body;  // first stage of a step: the input is read again as y
  const float term_i = lane_ok ? a.term[li] : 0.f;
  const C2 *zin_own = reinterpret_cast<const C2 *>(c.zin.body);
  C2 *out_own = reinterpret_cast<C2 *>(c.out.body);
  const C2 *y_own = reinterpret_cast<const C2 *>(c.y.body);
  const R *recs = reinterpret_cast<const R *>(c.recs_body);
  const int64_t rbase = c.rec_split;
  const int own0 = c.u_split;

  const int n_chunks = (c.u_end - c.u_begin + A - 1) / A;
  const int nwarps = gridDim.x * kTcWarps;
  const int first = blockIdx.x * kTcWarps + warp;
  const int cta_first = blockIdx.x * kTcWarps;
  // every warp of the CTA runs the same number of rounds (the tensor-core step is CTA-wide)
  const int n_rounds = (cta_first < n_chunks) ? (n_chunks - cta_first + nwarps - 1) / nwarps : 0;
  const int cap = 2 * S::RC;  // Hermitian runs: row-only slices
  auto load_offs = [&](int chn) -> int64_t {
    if (chn >= n_chunks) return 0;
    const int u0 = c.u_begin + chn * A;
    const int cnt = min(A, c.u_end - u0);
    return (lane <= cnt) ? c.link_off[u0 + lane] : (int64_t)0;
  };
  int64_t off_cur = load_offs(first);
  int64_t off_nxt = load_offs(first + nwarps);
  if (first < n_chunks) {
    const int u0 = c.u_begin + first * A;
    const int cnt = min(A, c.u_end - u0);
    issue_tiles<N, float, float>(zin_own, own0, u0, cnt, wb + W::tile0, lane, same_y);
    const int64_t lo = __shfl_sync(0xffffffffu, off_cur, 0), hi = __shfl_sync(0xffffffffu, off_cur, cnt);
    const int nr = heom_rec_batch(c.err, lo, (int)min(hi - lo, (int64_t)cap), rbase, c.n_recs);
    warp_copy16(wb + W::rec0, recs + (lo - rbase), nr * (int)sizeof(R), lane);
    cp_async_commit();
  }
  const uint32_t idesc = tf32_idesc(128, kTcK);
  const uint32_t my_ld = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes of D
  uint32_t phase = 0;
  int failed = 0;
  int pend_phase = -1;  // parity of a commit whose wait this thread gave up on (MMAs maybe in flight)
  int b = 0;
  for (int r = 0, chn = first; r < n_rounds; ++r, chn += nwarps, b ^= 1) {
    const bool valid = chn < n_chunks;  // warp-uniform
    const int u0 = c.u_begin + chn * A;
    const int cnt = valid ? min(A, c.u_end - u0) : 0;
    const int nx = chn + nwarps;
    const int64_t off_nx2 = load_offs(nx + nwarps);
    C2 *zt_all = reinterpret_cast<C2 *>(wb + (b ? W::tile1 : W::tile0));
    R *rec = reinterpret_cast<R *>(wb + (b ? W::rec1 : W::rec0));
    if (nx < n_chunks) {
      const int v0 = c.u_begin + nx * A;
      const int vcnt = min(A, c.u_end - v0);
      issue_tiles<N, float, float>(zin_own, own0, v0, vcnt, wb + (b ? W::tile0 : W::tile1), lane, same_y);
      const int64_t lo = __shfl_sync(0xffffffffu, off_nxt, 0), hi = __shfl_sync(0xffffffffu, off_nxt, vcnt);
      const int nr = heom_rec_batch(c.err, lo, (int)min(hi - lo, (int64_t)cap), rbase, c.n_recs);
      warp_copy16(wb + (b ? W::rec0 : W::rec1), recs + (lo - rbase), nr * (int)sizeof(R), lane);
    }
    cp_async_commit();
    if (valid && kYSmem && has_y) issue_tiles<N, float, float>(y_own, own0, u0, cnt, ybuf, lane);
    cp_async_commit();
    cp_async_wait<2>();  // this chunk's tiles and first records have landed
    __syncwarp();

    const bool active = valid && lane_ok && la < cnt;
    int64_t lo = 0, hi = 0;
    int nrec = 0;
    if (valid) {
      lo = __shfl_sync(0xffffffffu, off_cur, 0);
      hi = __shfl_sync(0xffffffffu, off_cur, cnt);
      nrec = (int)min(hi - lo, (int64_t)cap);
    }

    // own row s_{li, .} -> tensor-memory lane 32 warp + lane of the four A blocks (zeros for idle lanes)
    C2 zr[N];
    {
      const C2 *zt = zt_all + la * EPO;
      if (active) {
#pragma unroll
        for (int j = 0; j < N; ++j) zr[j] = zt[li * N + j];
      }
      // x = hi + lo: hi = x rounded to the 10 explicit mantissa bits of TF32 (add half a TF32 unit to
      // the magnitude bits, clear the 13 low bits), lo = x - hi exactly (|lo| <= 2^-11 |x|); the
      // tensor core reads lo's top 19 bits, so the split keeps about 21 bits of x
      uint32_t rh[kTcK], rl[kTcK], ih[kTcK], il[kTcK];
#pragma unroll
      for (int k = 0; k < kTcK; ++k) {
        const float xr = (k < N && active) ? zr[k < N ? k : 0].x : 0.f;
        const float xi = (k < N && active) ? zr[k < N ? k : 0].y : 0.f;
        rh[k] = (__float_as_uint(xr) + 0x1000u) & 0xFFFFE000u;
        ih[k] = (__float_as_uint(xi) + 0x1000u) & 0xFFFFE000u;
        rl[k] = __float_as_uint(xr - __uint_as_float(rh[k]));
        il[k] = __float_as_uint(xi - __uint_as_float(ih[k]));
      }
      tmem_st16(my_ld + kTcA + 0 * kTcK, rh);
      tmem_st16(my_ld + kTcA + 1 * kTcK, rl);
      tmem_st16(my_ld + kTcA + 2 * kTcK, ih);
      tmem_st16(my_ld + kTcA + 3 * kTcK, il);
      tmem_st_wait();
    }
    tc_fence_before();  // this warp's tensor-memory writes and reads precede the barrier
    failed = __syncthreads_or(failed);
    if (failed) break;
    if (threadIdx.x == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {
        const uint64_t bh = smem_desc(b_base + ks * 256, 128, 512);
        const uint64_t bl = smem_desc(b_base + TcSmem::b_tile + ks * 256, 128, 512);
#pragma unroll
        for (int part = 0; part < 2; ++part) {  // real, imaginary part of s
          const uint32_t d = tmem + part * kTcK;
          const uint32_t ah = tmem + kTcA + (2 * part) * kTcK + ks * 8;
          const uint32_t al = tmem + kTcA + (2 * part + 1) * kTcK + ks * 8;
          mma_tf32_ta(d, ah, bh, idesc, ks > 0 ? 1u : 0u);
          mma_tf32_ta(d, al, bh, idesc, 1u);
          mma_tf32_ta(d, ah, bl, idesc, 1u);
        }
      }
      mma_commit(mbar);
    }
    __syncwarp();

    // while the tensor cores run: neighbour gathers, half the decay and terminator (Q + Q^dagger
    // restores the rest), the links
    if (valid) issue_gathers<N, float, float>(c, rec, nrec, gbuf, lane);
    float rr[N], ri[N];
    if (active) {
      const float gsv = (float)c.gsum[u0 + la];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float f = 0.5f * (gsv + ((j != li) ? (term_i + a.term[j]) : 0.f));
        rr[j] = -f * zr[j].x;
        ri[j] = -f * zr[j].y;
      }
    }
    cp_async_wait<0>();  // gathers, y and the next chunk's copies have landed
    __syncwarp();
    if (valid)
      owner_apply<N, float, float>(c, recs, rbase, rec, gbuf, wb + W::tb, lo, hi, nrec, cap, u0, lane, rr, ri);

    {  // bounded wait for this round's MMAs
      const long long t0 = clock64();
      while (!mbar_try_wait(mbar, phase)) {
        if (clock64() - t0 > kTcWaitCycles) {
          failed = 1;
          pend_phase = (int)phase;
          break;
        }
      }
    }
    phase ^= 1u;
    failed = __any_sync(0xffffffffu, failed) ? 1 : 0;
    tc_fence_after();
    if (!failed) {
      uint32_t u[32];
      tmem_ld32(my_ld, u);
      if (active) {  // Q += i S
#pragma unroll
        for (int j = 0; j < N; ++j) {
          rr[j] -= __uint_as_float(u[kTcK + j]);
          ri[j] += __uint_as_float(u[j]);
        }
      }
    }
    if (valid) {
      owner_combine<N, float, float>(active, la, li, zt_all, rr, ri);
      __syncwarp();
      store_chunk<N, float, float>(out_own, y_own, own0, u0, cnt, has_y, a.ch, zt_all, ybuf, lane);
    }
    __syncwarp();  // this tile buffer, record buffer and ybuf are reused by later chunks
    off_cur = off_nxt;
    off_nxt = off_nx2;
  }
  cp_async_wait<0>();
  if (failed && threadIdx.x == 0 && c.err != nullptr) atomicOr(c.err, kErrTimeout);
  // Tensor memory must not be freed under MMAs that may still write it.  A thread that gave up on a
  // commit waits for it once more, again bounded; a thread whose wait on that commit succeeded saw
  // those MMAs complete.  Every thread that issued no wait after its last success has nothing in
  // flight: MMAs are issued only after the CTA barrier that precedes each round's wait.
  if (pend_phase >= 0) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, (uint32_t)pend_phase) && clock64() - t0 <= kTcWaitCycles) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc<kTcCols>(tmem);
  }
}

template <int N>
int launch_tc(const StageCommon &c, double ch, const double *term, const double *H, cudaStream_t st, int sm_count) {
  StageArgs<float> a;
  a.c = c;
  a.ch = (float)ch;
  for (int i = 0; i < kMaxStates; ++i) a.term[i] = (i < c.n) ? (float)term[i] : 0.f;
  for (int i = 0; i < kMaxStates * kMaxStates; ++i) {
    a.H[i] = 0.f;
    a.Hi[i] = 0.f;
  }
  for (int i = 0; i < c.n; ++i)
    for (int j = 0; j < c.n; ++j) a.H[i * kMaxStates + j] = (float)H[i * c.n + j];
  const size_t smem = (size_t)TcSmem::total + (size_t)kTcWarps * WarpSmem<N, float, float, kTcRC>::total;
  // CTAs per SM from the kernel's registers, shared memory and tensor memory (the occupancy API
  // answers 1 for kernels that allocate tensor memory; the persistent loop needs no co-residency, so
  // a count above what fits only queues CTAs)
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(stage_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, stage_tc_kernel<N>);
    int dev = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e != cudaSuccess) {
      set_error(std::string("tensor-core stage kernel: attributes: ") + cudaGetErrorString(e));
      return -4;
    }
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
    const int by_regs = regs_sm / (regs_warp * kTcWarps);
    const int by_smem = smem_sm / ((int)smem + smem_rsv);
    const int by_tmem = 512 / kTcCols;
    per_sm = std::min(std::min(by_regs, by_smem), by_tmem);
    if (per_sm < 1) {
      set_error("tensor-core stage kernel: does not fit on an SM");
      per_sm = 0;
      return -4;
    }
  }
  constexpr int A = StageShape<N, float, float>::A;
  const int n_chunks = (c.u_end - c.u_begin + A - 1) / A;
  const int blocks_needed = (n_chunks + kTcWarps - 1) / kTcWarps;
  const int grid = std::max(1, std::min(blocks_needed, sched_ctas(per_sm, c.occ_pct) * sm_count));
  stage_tc_kernel<N><<<grid, kTcWarps * 32, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("tensor-core stage kernel launch: ") + cudaGetErrorString(e));
    return -4;
  }
  return 0;
}

}  // namespace heom
