// Persistent warp-specialised tcgen05 contraction engine.
//
// A work item multiplies a 128-row tile of A with a tile of B (both K-major
// BF16 in global memory, read by TMA with 128-byte swizzle) in one or more
// "chunks"; a chunk is a run of 64-element k-blocks over one 128- or 256-row
// slice of B, accumulated in its own TMEM buffer (FP32, 128 lanes x TN
// columns). Buffers rotate through NBUF slots, so the epilogue of one chunk
// overlaps the MMAs of the next.
//
//   warp 0        TMA producer (one thread): ring of STAGES shared-memory stages
//   warp 1        MMA issuer (one thread)
//   warps 2..5    epilogue; thread = TMEM lane = row of the A tile
//
// SPLIT = 3 multiplies two-part operands (x = hi + lo, both BF16):
// hi*hi + hi*lo + lo*hi. SPLIT = 2 multiplies a two-part A with a B that is
// exact in BF16 (hi*b + lo*b). Chunking the reduction dimension bounds how many
// MMA steps feed one accumulator: the tensor-core FP32 accumulation is not
// round-to-nearest, and the chunk partials are summed in FP32 on the CUDA
// cores by the epilogue.
//
// Optionally (ACCS > 1) a chunk has several accumulators side by side in TMEM
// (accumulator a at column a * TN of the chunk's buffer) and the policy routes
// each product of each k-block to one of them:
//   static constexpr int ACCS;
//   static int acc_of(int product, int kb_in_chunk, int kbs_in_chunk);   (product: 0 hi*hi, 1 hi*lo, 2 lo*hi)
//
// A policy class P supplies the schedule and the epilogue:
//   static constexpr int TN, NBUF, STAGES, SPLIT, EB;          (EB: operand bytes, 2 BF16 / 1 E4M3)
//   struct Item; struct Ctx;                                  (per-thread epilogue state)
//   int64_t total() const;  Item decode(int64_t) const;
//   int nchunks(const Item&) const;
//   void chunk(const Item&, int c, int& b_row, int& kb0, int& kb1) const;
//   int a_row(const Item&) const;
//   void epi_begin(const Item&, Ctx&, int m, int ew, uint8_t* warp_smem) const;
//   void epi_chunk(const Item&, int c, uint32_t taddr, Ctx&, int m, uint8_t* warp_smem) const;
//   void epi_end(const Item&, Ctx&, int m, uint8_t* warp_smem) const;
//   static constexpr int kWarpSmem;                           (bytes per epilogue warp)
// Optionally (GEN_A = true) the A operand is not loaded by TMA but written
// into the stage (128-byte swizzled, K-major) by GEN_WARPS generator warps:
// warp 0 and warps 6 .. 4 + GEN_WARPS; generator thread g = 32 * (generator
// warp) + lane, g < 32 * GEN_WARPS. Lane 0 of warp 0 starts the B copy as
// soon as a stage is free; each generator warp arrives on the stage's full
// barrier once its part of the A tile is written.
//   static constexpr int GEN_WARPS;                           (1 .. 4)
//   struct GenRegs;          (per-thread loads of one k-block: gen_load only issues them, and nothing reads
//                             them before gen_store two k-blocks later, so their latency is hidden)
//   struct GenPos;           (the tile entries a thread wrote)
//   void gen_load(const Item&, int kb, int g, GenRegs&) const;
//   void gen_store(const Item&, int kb, int g, const GenRegs&, const GenPos* prev, GenPos& now, uint8_t* a_hi,
//                  uint8_t* a_lo) const;             (prev: what this stage held last time, null on first use)
// The engine zeroes every stage's A tiles before the first k-block.
#pragma once
#include <type_traits>

#include "tc_common.cuh"

namespace gift {
namespace tc {

constexpr int kTM = 128;
constexpr int kTK = 64;
constexpr int kEngineThreads = 192;

template <class P, class = void>
struct gen_a_of : std::false_type {};
template <class P>
struct gen_a_of<P, std::void_t<decltype(P::GEN_A)>> : std::integral_constant<bool, P::GEN_A> {};

template <class P, class = void>
struct gen_warps_of : std::integral_constant<int, 1> {};
template <class P>
struct gen_warps_of<P, std::void_t<decltype(P::GEN_WARPS)>> : std::integral_constant<int, P::GEN_WARPS> {};

// SWAP_CROSS = true: with SPLIT = 3 the two cross products of a k-block are
// issued as lo(A) * hi(B) before hi(A) * lo(B), so that an engine run with the
// operand roles exchanged accumulates the same products in the same order
template <class P, class = void>
struct swap_cross_of : std::false_type {};
template <class P>
struct swap_cross_of<P, std::void_t<decltype(P::SWAP_CROSS)>> : std::integral_constant<bool, P::SWAP_CROSS> {};

template <class P, class = void>
struct accs_of : std::integral_constant<int, 1> {};
template <class P>
struct accs_of<P, std::void_t<decltype(P::ACCS)>> : std::integral_constant<int, P::ACCS> {};

// EPI_SPLIT = 2 or 4: 4 * EPI_SPLIT epilogue warps, EPI_SPLIT per TMEM lane
// quadrant, each taking 1 / EPI_SPLIT of the tile's columns (policy argument
// ew = warp - 2, column part ew / 4)
template <class P, class = void>
struct epi_split_of : std::integral_constant<int, 1> {};
template <class P>
struct epi_split_of<P, std::void_t<decltype(P::EPI_SPLIT)>> : std::integral_constant<int, P::EPI_SPLIT> {};

// threads of the engine CTA: producer, MMA, epilogue warps, extra generator warps
template <class P>
struct engine_threads
    : std::integral_constant<int, kEngineThreads + 128 * (epi_split_of<P>::value - 1) +
                                      (gen_a_of<P>::value ? 32 * (gen_warps_of<P>::value - 1) : 0)> {};

template <class P>
struct EngineLayout {
  // one k-block = one 128-byte swizzle row of K: 64 BF16 or 128 E4M3 elements
  static constexpr int kKElems = 128 / P::EB;
  static constexpr int kABytes = kTM * 128;
  static constexpr int kBBytes = P::TN * 128;
  static_assert(P::EB == 2 || P::SPLIT == 1, "two-part operands are BF16");
  static_assert(P::SPLIT == 1 || P::SPLIT == 2 || P::SPLIT == 3, "SPLIT is 1, 2 or 3");
  static constexpr int kPartsA = P::SPLIT == 1 ? 1 : 2;
  static constexpr int kPartsB = P::SPLIT == 3 ? 2 : 1;
  // stage: A, B, then (two-part) A lo, then (SPLIT 3) B lo
  static constexpr int kStageBytes = kPartsA * kABytes + kPartsB * kBBytes;
  static constexpr int kBarBytes = 256;  // full/empty per stage, full/empty per TMEM buffer, then the TMEM address
  static_assert((2 * P::STAGES + 2 * P::NBUF) * 8 + 4 <= kBarBytes, "barriers and TMEM address fit in 256 bytes");
  static constexpr int kEpiWarps = 4 * epi_split_of<P>::value;
  static_assert(epi_split_of<P>::value == 1 || epi_split_of<P>::value == 2 || epi_split_of<P>::value == 4,
                "EPI_SPLIT is 1, 2 or 4");
  static_assert(epi_split_of<P>::value == 1 || !gen_a_of<P>::value, "generated A tiles take four epilogue warps");
  static constexpr int kSmem = 1024 + P::STAGES * kStageBytes + kBarBytes + kEpiWarps * P::kWarpSmem;
  static constexpr int kAccs = accs_of<P>::value;
  static_assert(P::NBUF * kAccs * P::TN <= 512, "TMEM holds 512 columns");
  static_assert(kSmem <= 232448, "shared memory per CTA");
};

template <class P>
__global__ void __launch_bounds__(engine_threads<P>::value, 1)
    tc_engine(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2, const P p,
              int* err) {
  using L = EngineLayout<P>;
  constexpr int S = P::STAGES;
  constexpr int NB = P::NBUF;
  constexpr int TN = P::TN;
  constexpr bool kGen = gen_a_of<P>::value;
  constexpr int kGenWarps = kGen ? gen_warps_of<P>::value : 1;
  static_assert(kGenWarps >= 1 && kGenWarps <= 4, "one to four generator warps");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tiles = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * L::kStageBytes);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * S + 2 * NB);
  uint8_t* wsm = smem + S * L::kStageBytes + L::kBarBytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * S;
  const uint32_t tfull0 = empty0 + 8 * S;
  const uint32_t tempty0 = tfull0 + 8 * NB;
  constexpr int kAccs = L::kAccs;
  constexpr int kBufCols = kAccs * TN;  // TMEM columns of one chunk buffer
  constexpr uint32_t kCols = (NB * kBufCols <= 32) ? 32 : (NB * kBufCols <= 64) ? 64 : (NB * kBufCols <= 128) ? 128
                             : (NB * kBufCols <= 256) ? 256 : 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, kGenWarps);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, L::kEpiWarps);
    }
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_holder), kCols);
    tmem_relinquish();
  }
  if constexpr (kGen) {  // generated A tiles start as zeros
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int s = 0; s < S; ++s) {
      uint8_t* st = tiles + s * L::kStageBytes;
      for (int o = threadIdx.x * 16; o < L::kABytes; o += engine_threads<P>::value * 16) {
        *reinterpret_cast<uint4*>(st + o) = z;
        if (L::kPartsA == 2) *reinterpret_cast<uint4*>(st + L::kABytes + L::kBBytes + o) = z;
      }
    }
    fence_proxy_async_smem();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  const int64_t total = p.total();
  constexpr uint32_t kIdesc = P::EB == 2 ? idesc_bf16(kTM, TN) : idesc_e4m3(kTM, TN);
  constexpr int KE = L::kKElems;

  if (warp == 0 || (kGen && warp >= 6)) {
    if constexpr (kGen) {
      // every generator thread writes its part of the A tile of every k-block,
      // with the loads for the next two k-blocks in flight; lane 0 of warp 0
      // loads B by TMA
      const int gw = warp == 0 ? 0 : warp - 5;
      const int gt = gw * 32 + lane;
      const bool tma_lane = gw == 0 && lane == 0;
      if (tma_lane) prefetch_tmap(&tmB);
      struct Cur {
        int64_t item;
        typename P::Item it;
        int nch, c, kb, kb1, br;
        bool valid;
      };
      auto seek = [&](Cur& x) {  // first k-block at or after x.kb
        while (x.valid && x.kb >= x.kb1) {
          if (++x.c < x.nch) {
            p.chunk(x.it, x.c, x.br, x.kb, x.kb1);
          } else {
            x.item += gridDim.x;
            if (x.item >= total) {
              x.valid = false;
            } else {
              x.it = p.decode(x.item);
              x.nch = p.nchunks(x.it);
              x.c = 0;
              p.chunk(x.it, 0, x.br, x.kb, x.kb1);
            }
          }
        }
      };
      Cur c0;
      c0.item = blockIdx.x;
      c0.valid = c0.item < total;
      c0.c = 0;
      c0.kb = c0.kb1 = 0;
      c0.nch = 0;
      c0.br = 0;
      if (c0.valid) {
        c0.it = p.decode(c0.item);
        c0.nch = p.nchunks(c0.it);
        p.chunk(c0.it, 0, c0.br, c0.kb, c0.kb1);
        seek(c0);
      }
      Cur c1 = c0;
      if (c1.valid) {
        ++c1.kb;
        seek(c1);
      }
      Cur c2 = c1;
      if (c2.valid) {
        ++c2.kb;
        seek(c2);
      }
      // three register sets rotate by name, so the loads for a k-block are
      // issued two k-blocks before their values are used (no copies between)
      typename P::GenRegs ga, gb, gc;
      // what each stage's A tile holds (its previous k-block): the loop below
      // visits stages 0, 1, 2 in its three calls, so each call names its own
      // record and the records stay in registers
      static_assert(S == 3, "generated A tiles rotate through three stages");
      typename P::GenPos held0, held1, held2;
      bool used0 = false, used1 = false, used2 = false;
      if (c0.valid) p.gen_load(c0.it, c0.kb, gt, ga);
      if (c1.valid) p.gen_load(c1.it, c1.kb, gt, gb);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int last_phase[S];
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) last_phase[s2] = -1;
      constexpr uint32_t kBTx = L::kPartsB * L::kBBytes;
      // one k-block: prefetch into `fill` for c2, write c0's tile from `use`
      auto step = [&](typename P::GenRegs& use, typename P::GenRegs& fill, typename P::GenPos& held,
                      bool& used) -> bool {
        if (!ok || !c0.valid) return false;
        if (c2.valid) p.gen_load(c2.it, c2.kb, gt, fill);
        int w_ok = 1;
        if (lane == 0) w_ok = mbar_wait(empty0 + 8 * stage, phase ^ 1, err, kErrProducer) ? 1 : 0;
        w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
        if (!w_ok) {
          ok = false;
          return false;
        }
        uint8_t* st = tiles + stage * L::kStageBytes;
        if (tma_lane) {  // B is in flight while the A tile is written
          const uint32_t sa = smem_u32(st);
          mbar_expect_tx_only(full0 + 8 * stage, kBTx);
          tma_load_2d(sa + L::kABytes, &tmB, c0.kb * KE, c0.br, full0 + 8 * stage);
          if (P::SPLIT == 3)
            tma_load_2d(sa + 2 * L::kABytes + L::kBBytes, &tmB2, c0.kb * KE, c0.br, full0 + 8 * stage);
          last_phase[stage] = (int)phase;
        }
        typename P::GenPos now;
        p.gen_store(c0.it, c0.kb, gt, use, used ? &held : nullptr, now, st, st + L::kABytes + L::kBBytes);
        held = now;
        used = true;
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(full0 + 8 * stage);
        if (++stage == S) {
          stage = 0;
          phase ^= 1;
        }
        c0 = c1;
        c1 = c2;
        if (c2.valid) {
          ++c2.kb;
          seek(c2);
        }
        return true;
      };
      while (step(ga, gc, held0, used0) && step(gb, ga, held1, used1) && step(gc, gb, held2, used2)) {
      }
      if (!ok && tma_lane) {
        for (int s2 = 0; s2 < S; ++s2) {  // let issued copies land before exiting (bounded)
          if (last_phase[s2] < 0) continue;
          const long long t0 = clock64();
          while (!mbar_try_wait(full0 + 8 * s2, (uint32_t)last_phase[s2]) && clock64() - t0 < kWaitCycles / 4) {
          }
        }
      }
      __syncwarp();
    } else {
      if (lane == 0) {
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        int last_phase[S];
#pragma unroll
        for (int s = 0; s < S; ++s) last_phase[s] = -1;
        for (int64_t item = blockIdx.x; ok && item < total; item += gridDim.x) {
          const typename P::Item it = p.decode(item);
          const int ar = p.a_row(it);
          const int nch = p.nchunks(it);
          for (int c = 0; ok && c < nch; ++c) {
            int br, kb0, kb1;
            p.chunk(it, c, br, kb0, kb1);
            for (int kb = kb0; kb < kb1; ++kb) {
              if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, err, kErrProducer)) {
                ok = false;
                break;
              }
              const uint32_t st = smem_u32(tiles + stage * L::kStageBytes);
              mbar_expect_tx(full0 + 8 * stage, L::kStageBytes);
              tma_load_2d(st, &tmA, kb * KE, ar, full0 + 8 * stage);
              tma_load_2d(st + L::kABytes, &tmB, kb * KE, br, full0 + 8 * stage);
              if (P::SPLIT >= 2) tma_load_2d(st + L::kABytes + L::kBBytes, &tmA2, kb * KE, ar, full0 + 8 * stage);
              if (P::SPLIT == 3) tma_load_2d(st + 2 * L::kABytes + L::kBBytes, &tmB2, kb * KE, br, full0 + 8 * stage);
              last_phase[stage] = (int)phase;
              if (++stage == S) {
                stage = 0;
                phase ^= 1;
              }
            }
          }
        }
        if (!ok) {
          for (int s = 0; s < S; ++s) {  // let issued copies land before exiting (bounded)
            if (last_phase[s] < 0) continue;
            const long long t0 = clock64();
            while (!mbar_try_wait(full0 + 8 * s, (uint32_t)last_phase[s]) && clock64() - t0 < kWaitCycles / 4) {
            }
          }
        }
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int buf = 0;
      uint32_t bphase = 0;
      for (int64_t item = blockIdx.x; ok && item < total; item += gridDim.x) {
        const typename P::Item it = p.decode(item);
        const int nch = p.nchunks(it);
        for (int c = 0; ok && c < nch; ++c) {
          int br, kb0, kb1;
          p.chunk(it, c, br, kb0, kb1);
          if (!mbar_wait(tempty0 + 8 * buf, bphase ^ 1, err, kErrMma)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t d = tmem + buf * kBufCols;
          uint32_t written = 0;  // accumulators of this chunk written so far (kAccs > 1)
          (void)written;
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(full0 + 8 * stage, phase, err, kErrMma)) {
              ok = false;
              break;
            }
            fence_after_sync();
            const uint32_t sa = smem_u32(tiles + stage * L::kStageBytes);
            const uint32_t sb = sa + L::kABytes;
            const uint32_t sa2 = sb + L::kBBytes;
            const uint32_t sb2 = sa2 + L::kABytes;
            // four MMAs of 32 bytes of K each (16 BF16 or 32 E4M3 elements)
            if constexpr (kAccs == 1) {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc_in = (kb != kb0 || kk != 0) ? 1u : 0u;
                if (P::EB == 1) {
                  mma_f8(d, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), kIdesc, acc_in);
                  continue;
                }
                mma_f16(d, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), kIdesc, acc_in);
                if (swap_cross_of<P>::value && P::SPLIT == 3) {
                  mma_f16(d, sdesc_sw128(sa2 + kk * 32), sdesc_sw128(sb + kk * 32), kIdesc, 1u);
                  mma_f16(d, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb2 + kk * 32), kIdesc, 1u);
                  continue;
                }
                if (P::SPLIT == 3) mma_f16(d, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb2 + kk * 32), kIdesc, 1u);
                if (P::SPLIT >= 2) mma_f16(d, sdesc_sw128(sa2 + kk * 32), sdesc_sw128(sb + kk * 32), kIdesc, 1u);
              }
            } else {
              static_assert(P::EB == 2, "routed accumulators take BF16 products");
              const int a0 = P::acc_of(0, kb - kb0, kb1 - kb0);
              const int a1 = P::acc_of(1, kb - kb0, kb1 - kb0);
              const int a2 = P::acc_of(2, kb - kb0, kb1 - kb0);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                mma_f16(d + a0 * TN, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), kIdesc,
                        (written >> a0) & 1u);
                written |= 1u << a0;
                if (P::SPLIT == 3) {
                  mma_f16(d + a1 * TN, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb2 + kk * 32), kIdesc,
                          (written >> a1) & 1u);
                  written |= 1u << a1;
                }
                if (P::SPLIT >= 2) {
                  mma_f16(d + a2 * TN, sdesc_sw128(sa2 + kk * 32), sdesc_sw128(sb + kk * 32), kIdesc,
                          (written >> a2) & 1u);
                  written |= 1u << a2;
                }
              }
            }
            mma_commit(empty0 + 8 * stage);
            if (++stage == S) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          mma_commit(tfull0 + 8 * buf);
          if (++buf == NB) {
            buf = 0;
            bphase ^= 1;
          }
        }
      }
    }
    __syncwarp();
  } else if (warp < 2 + L::kEpiWarps) {
    const int quad = warp & 3;
    const int m = quad * 32 + lane;
    const int ew = warp - 2;
    uint8_t* my = wsm + ew * P::kWarpSmem;
    int buf = 0;
    uint32_t bphase = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; ok && item < total; item += gridDim.x) {
      const typename P::Item it = p.decode(item);
      typename P::Ctx ctx;
      __syncwarp();
      p.epi_begin(it, ctx, m, ew, my);
      __syncwarp();
      const int nch = p.nchunks(it);
      for (int c = 0; c < nch; ++c) {
        if (!mbar_wait(tfull0 + 8 * buf, bphase, err, kErrTmemFull)) {
          ok = false;
          break;
        }
        fence_after_sync();
        p.epi_chunk(it, c, tmem + (static_cast<uint32_t>(quad * 32) << 16) + buf * kBufCols, ctx, m, my);
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
        if (++buf == NB) {
          buf = 0;
          bphase ^= 1;
        }
      }
      if (!ok) break;
      p.epi_end(it, ctx, m, my);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tmem, kCols);
  }
}

// Launch on every SM of the current device (persistent CTAs).
template <class P>
void launch_engine(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& a2, const CUtensorMap& b2,
                   const P& p, int* err, int grid, cudaStream_t s) {
  using L = EngineLayout<P>;
  GIFT_CUDA(cudaFuncSetAttribute(tc_engine<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem));
  tc_engine<P><<<grid, engine_threads<P>::value, L::kSmem, s>>>(a, b, a2, b2, p, err);
  GIFT_LAUNCHED("tc_engine");
}

}  // namespace tc
}  // namespace gift
