// S-IF re-ranking that allocates no device memory.
//
// Some callers cannot allocate device memory when they re-rank: a process
// whose free device memory is entirely reserved by another allocator (a
// serving framework's caching pool) would see the allocation fail, and a
// latency-critical loop must not enter the CUDA allocator at all (freeing
// device memory can synchronise the device). For them, gift_rerank_noalloc
// runs the same re-ranking kernels as gift_rerank on one fixed scratch
// buffer that lives in this file as a device variable: it is created with
// the library's module on every device that uses it and is held until the
// process exits.
//
// Host code cannot use the name of a __device__ variable as an address; the
// first call on each device asks the runtime for the variable's device
// address (with that device current) and remembers it. Later calls check that
// the remembered address is still a device allocation of that device (after a
// cudaDeviceReset the module, and with it the buffer, is loaded anew) and look
// it up again when it is not.
#include <mutex>

#include "gift_internal.cuh"

namespace gift {

namespace {

constexpr size_t kScratchBytes = (size_t)GIFT_RERANK_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_rerank_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<void*> g_addr;  // device address of g_rerank_scratch per device ordinal

bool still_valid(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

void* scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev] || !still_valid(g_addr[dev], dev)) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rerank_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      fail(GIFT_ECUDA, std::string("cannot get the device address of the re-rank scratch: ") +
                           cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace gift

extern "C" gift_status gift_rerank_noalloc(gift_index* index, const int32_t* cand_ids, const float* cand_scores,
                                           int32_t B, int32_t n_cand, int32_t k1, int32_t topk, int32_t* out_ids,
                                           float* out_sprime, cudaStream_t stream) {
  return gift::guarded("gift_rerank_noalloc", [&] {
    GIFT_REQUIRE(index && cand_ids && cand_scores && out_ids && out_sprime, "NULL argument");
    const gift::Index& ix = *reinterpret_cast<const gift::Index*>(index);
    if (!ix.ready()) gift::fail(GIFT_ESTATE, "the streamed build of this index is not complete");
    if (!ix.sif_off) gift::fail(GIFT_EUNSUPPORTED, "index built without an S-IF (sif_k1 == 0)");
    int dev = 0;
    GIFT_CUDA(cudaGetDevice(&dev));
    GIFT_REQUIRE(dev == ix.device, "gift_rerank_noalloc must be called with the index's device current");
    GIFT_REQUIRE(B > 0 && n_cand > 0 && k1 > 0 && k1 <= n_cand, "need 0 < k1 <= n_cand and B > 0");
    GIFT_REQUIRE(topk > 0 && topk <= 1024, "topk must be in [1, 1024]");
    GIFT_REQUIRE(gift::on_device(cand_ids) && gift::on_device(cand_scores) && gift::on_device(out_ids) &&
                     gift::on_device(out_sprime),
                 "gift_rerank_noalloc takes device buffers only (host buffers would need staging memory)");
    const size_t need = gift::sif_rerank_scratch_bytes(B, ix.sif_n, topk);
    if (need > gift::kScratchBytes)
      gift::fail(GIFT_EINVAL, "gift_rerank_noalloc needs " + std::to_string(need) +
                                  " bytes of scratch for this batch; its fixed buffer holds " +
                                  std::to_string(gift::kScratchBytes) + " bytes: split the batch");
    void* scratch = gift::scratch_address(dev);
    gift::sif_rerank_into(ix, cand_ids, cand_scores, B, n_cand, k1, topk, out_ids, out_sprime, scratch,
                          gift::kScratchBytes, stream);
  });
}
