// Host helpers of the tcgen05 kernels: TMA tensor maps and device queries.
#include "tc_common.cuh"

namespace gift {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver entry point is fetched through the runtime, so the library does
// not link against the driver library and still loads on GPU-less hosts
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    GIFT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) fail(GIFT_ECUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

CUtensorMap make_tmap_bf16(const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows, uint64_t pitch) {
  if (pitch == 0) pitch = cols;
  GIFT_REQUIRE(reinterpret_cast<uintptr_t>(base) % 16 == 0, "tensor map base must be 16-byte aligned");
  GIFT_REQUIRE((pitch * 2) % 16 == 0 && pitch >= cols, "tensor map row pitch must be >= cols and a multiple of 16 bytes");
  GIFT_REQUIRE(box_rows >= 1 && box_rows <= 256, "tensor map box rows must be in [1, 256]");
  // callers pad every source by one box, so a tile never leaves the allocation
  GIFT_REQUIRE(rows >= box_rows, "tensor map extent must cover at least one box");
  CUtensorMap m;
  const cuuint64_t dims[2] = {cols, rows > 0 ? rows : 1};
  const cuuint64_t strides[1] = {pitch * 2};
  const cuuint32_t box[2] = {64u, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(GIFT_ECUDA, "cuTensorMapEncodeTiled failed with " + std::to_string((int)r));
  return m;
}

CUtensorMap make_tmap_u8(const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows, uint64_t pitch) {
  if (pitch == 0) pitch = cols;
  GIFT_REQUIRE(reinterpret_cast<uintptr_t>(base) % 16 == 0, "tensor map base must be 16-byte aligned");
  GIFT_REQUIRE(pitch % 16 == 0 && pitch >= cols, "tensor map row pitch must be >= cols and a multiple of 16 bytes");
  GIFT_REQUIRE(box_rows >= 1 && box_rows <= 256, "tensor map box rows must be in [1, 256]");
  GIFT_REQUIRE(rows >= box_rows, "tensor map extent must cover at least one box");
  CUtensorMap m;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {pitch};
  const cuuint32_t box[2] = {128u, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(GIFT_ECUDA, "cuTensorMapEncodeTiled failed with " + std::to_string((int)r));
  return m;
}

int device_sm_count() {
  int dev = 0, n = 0;
  GIFT_CUDA(cudaGetDevice(&dev));
  GIFT_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n;
}

}  // namespace gift
