// Page-locked host buffers backed by transparent huge pages (lbm_host_alloc,
// lbm_host_free).  The paper has no counterpart; this is a deployment helper
// for the host arrays that the C ABI copies to and from the device.
//
// A DMA copy between the GPU and host memory translates every host page it
// touches.  Anonymous memory advised for transparent huge pages is mapped in
// large blocks wherever the kernel can provide them, and stays so on hosts
// whose memory has been fragmented by earlier jobs, where small-page pinned
// buffers (cudaHostAlloc) were measured to copy several times below the link
// rate.
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <unistd.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "lbm.h"

namespace {

struct Mapping {
  void* raw;        // start of the anonymous mapping
  size_t raw_len;   // its length
  size_t len;       // registered length from the aligned start
};

std::mutex g_mutex;
std::map<void*, Mapping> g_buffers;  // aligned start -> mapping

// Transparent huge-page size of this kernel (PMD size), else 2 MiB.
size_t huge_page_size() {
  size_t hp = size_t(2) << 20;
  if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long v = 0;
    if (std::fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) hp = size_t(v);
    std::fclose(f);
  }
  return hp;
}

}  // namespace

extern "C" lbm_status lbm_host_alloc(size_t bytes, void** out) {
  if (!out || bytes == 0) return LBM_E_INVAL;
  *out = nullptr;
  if (bytes > (~size_t(0) >> 2)) return LBM_E_INVAL;
  // Buffers of at least one huge page are aligned to and rounded up to huge
  // pages (the huge page is 2 MiB with 4 KiB base pages, 512 MiB with
  // 64 KiB ones); smaller ones keep base pages, so they cost no more than
  // their size.
  const size_t page = size_t(sysconf(_SC_PAGESIZE));
  const size_t hp = huge_page_size();
  const size_t unit = bytes >= hp ? hp : page;
  const size_t len = (bytes + unit - 1) / unit * unit;
  const size_t raw_len = unit == hp ? len + hp : len;  // room to align the start
  void* raw = mmap(nullptr, raw_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return LBM_E_NOMEM;
  const uintptr_t a = (reinterpret_cast<uintptr_t>(raw) + unit - 1) / unit * unit;
  char* p = reinterpret_cast<char*>(a);
  if (unit == hp) (void)madvise(p, len, MADV_HUGEPAGE);  // advisory: base pages where refused
  // fault the range in, one allocation unit at a time (zero-filled)
  for (size_t off = 0; off < len; off += unit) p[off] = 0;
  if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(raw, raw_len);
    return LBM_E_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    g_buffers[p] = Mapping{raw, raw_len, len};
  }
  *out = p;
  return LBM_OK;
}

extern "C" lbm_status lbm_host_free(void* p) {
  if (!p) return LBM_OK;
  Mapping m;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    const auto it = g_buffers.find(p);
    if (it == g_buffers.end()) return LBM_E_INVAL;
    m = it->second;
    g_buffers.erase(it);
  }
  const cudaError_t e = cudaHostUnregister(p);
  if (e != cudaSuccess) cudaGetLastError();
  munmap(m.raw, m.raw_len);
  return e == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}
