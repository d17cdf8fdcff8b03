// Host side of the engine GEMM (instantiations of GemmPolicy).
#include "tc_gemm.cuh"

namespace gift {

void gemm_tc(const __nv_bfloat16* a_hi, const __nv_bfloat16* a_lo, int64_t M, int64_t a_rows_alloc, int64_t lda,
             const __nv_bfloat16* b_hi, const __nv_bfloat16* b_lo, int64_t N, int64_t b_rows_alloc, int64_t ldb, int K,
             float* C, int64_t ldc, int accumulate, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  const bool split = a_lo != nullptr && b_lo != nullptr;
  const CUtensorMap tA = make_tmap_bf16(a_hi, a_rows_alloc, K, tc::kTM, lda);
  const CUtensorMap tB = make_tmap_bf16(b_hi, b_rows_alloc, K, 128, ldb);
  const int sms = device_sm_count();
  if (split) {
    GemmPolicy<3> p;
    p.M = M;
    p.N = N;
    p.nkb = (int)cdiv(K, tc::kTK);
    p.C = C;
    p.ldc = ldc;
    p.accumulate = accumulate;
    const CUtensorMap tA2 = make_tmap_bf16(a_lo, a_rows_alloc, K, tc::kTM, lda);
    const CUtensorMap tB2 = make_tmap_bf16(b_lo, b_rows_alloc, K, 128, ldb);
    const int grid = (int)std::min<int64_t>(sms, cdiv(M, tc::kTM) * cdiv(N, 128));
    tc::launch_engine(tA, tB, tA2, tB2, p, err, grid, s);
  } else {
    GemmPolicy<1> p;
    p.M = M;
    p.N = N;
    p.nkb = (int)cdiv(K, tc::kTK);
    p.C = C;
    p.ldc = ldc;
    p.accumulate = accumulate;
    const int grid = (int)std::min<int64_t>(sms, cdiv(M, tc::kTM) * cdiv(N, 128));
    tc::launch_engine(tA, tB, tA, tB, p, err, grid, s);
  }
}

}  // namespace gift
