// Tile-key sort that allocates nothing: the stable radix sort of the tile
// binning stage with its working memory in a file-scope device array.
//
// Who needs it: callers that may not allocate device memory once they are
// running, e.g. a host renderer or robot stack that reserves every byte of
// the GPU up front under its own allocator, or code on a latency-critical
// path where a cudaMalloc (which can synchronise the device) is not
// allowed. They pass their own input and output buffers; the working memory
// this call needs comes from a fixed array that the library image carries.
#include <mutex>

#include "nbv_internal.cuh"

namespace nbv {
int launch_radix_pass(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                      int64_t count, int shift, uint32_t* hist, cudaStream_t st);
}  // namespace nbv

namespace {

constexpr int64_t kMaxPairs = NBV_NOALLOC_MAX_PAIRS;
// radix histograms for kMaxPairs keys: 2 x 256 x ceil(kMaxPairs / 2048) words (the
// radix tile holds at least 2048 keys)
// plus the block sums of their scan (ceil(. / 4096) + 64 words)
constexpr int64_t kBlocks = (kMaxPairs + 2047) / 2048;
constexpr int64_t kHistWords = 2 * 256 * kBlocks + (256 * kBlocks + 4095) / 4096 + 64;
constexpr size_t kKeyBytes = sizeof(uint64_t) * (size_t)kMaxPairs;
constexpr size_t kValBytes = sizeof(uint32_t) * (size_t)kMaxPairs;
constexpr size_t kHistBytes = sizeof(uint32_t) * (size_t)kHistWords;
constexpr size_t kScratchBytes = kKeyBytes + kValBytes + kHistBytes;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Whether the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" int nbv_sort_tile_keys_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, int64_t n,
                                          int key_bits, uint64_t* keys_out, uint32_t* vals_out,
                                          void* cuda_stream) {
  if (n < 0 || n > kMaxPairs || key_bits < 1 || key_bits > 64) return NBV_ERR_ARG;
  if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return NBV_ERR_ARG;
  if (n > 0) {
    // the outputs may share no byte with the inputs or with each other
    const size_t kb = sizeof(uint64_t) * (size_t)n, vb = sizeof(uint32_t) * (size_t)n;
    if (overlap(keys_out, kb, keys_in, kb) || overlap(keys_out, kb, vals_in, vb) ||
        overlap(vals_out, vb, keys_in, kb) || overlap(vals_out, vb, vals_in, vb) ||
        overlap(keys_out, kb, vals_out, vb))
      return NBV_ERR_ARG;
  }
  // a launch error left pending by earlier work on this thread is cleared
  // here, so that the check after this call's launches reports only its own
  cudaGetLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NBV_ERR_CUDA;
  void* base = nullptr;
  {
    // set-up, once per device: the device address of the array (the host-side
    // symbol is only a stand-in and must never reach a kernel)
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return NBV_ERR_CUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    base = g_scratch_ptr[dev];
  }
  if (n == 0) return NBV_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  uint64_t* ks = reinterpret_cast<uint64_t*>(b);
  uint32_t* vs = reinterpret_cast<uint32_t*>(b + kKeyBytes);
  uint32_t* hist = reinterpret_cast<uint32_t*>(b + kKeyBytes + kValBytes);
  const int passes = (key_bits + 7) / 8;
  // ping-pong between the scratch copy and the caller's output so that the
  // last pass lands in the output; the input is only read
  const uint64_t* kin = keys_in;
  const uint32_t* vin = vals_in;
  for (int p = 0; p < passes; ++p) {
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint64_t* kout = to_out ? keys_out : ks;
    uint32_t* vout = to_out ? vals_out : vs;
    nbv::launch_radix_pass(kin, vin, kout, vout, n, 8 * p, hist, st);
    kin = kout;
    vin = vout;
  }
  if (cudaGetLastError() != cudaSuccess) return NBV_ERR_CUDA;
  return NBV_OK;
}
