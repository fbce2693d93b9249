// Device memory for libctd from PyTorch's CUDA caching allocator.
//
// The two functions below are handed to ctd_set_allocator (include/ctd.h)
// by the Python binding, so that every device allocation of the library
// comes from the same caching allocator as the caller's tensors: memory
// the library frees is reused by PyTorch and the other way round, and
// torch.cuda.memory_allocated() counts what the library holds.  They call
// the allocator's C++ entry points directly (no Python per allocation).
#include <c10/cuda/CUDACachingAllocator.h>
#include <cuda_runtime.h>

#include <cstddef>

extern "C" __attribute__((visibility("default"))) void* ctd_torch_alloc(size_t bytes,
                                                                        void* stream) {
  try {
    return c10::cuda::CUDACachingAllocator::raw_alloc_with_stream(
        bytes, static_cast<cudaStream_t>(stream));
  } catch (...) {
    return nullptr;  // out of memory: the library reports CTD_ENOMEM
  }
}

// The caching allocator frees in the order of the stream the block was
// allocated on, which is the stream the library releases it on.
extern "C" __attribute__((visibility("default"))) void ctd_torch_release(void* ptr,
                                                                         void* stream) {
  (void)stream;
  try {
    c10::cuda::CUDACachingAllocator::raw_delete(ptr);
  } catch (...) {
  }
}
