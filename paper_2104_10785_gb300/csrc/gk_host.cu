// gk_host.cu -- pinned host buffers for operands and results that stay fast to copy.
//
// On a Grace host the GPU reaches pinned host pages through the host's address
// translation; with the default 64 KB pages an 8 GB buffer is 131 072 translations,
// and after long kernel runs the first full copy of such a buffer measured 25-100 GB/s
// instead of 210 GB/s.  A buffer backed by transparent huge pages (one translation per
// huge page) copied at 210 GB/s every time.  gk_host_alloc maps anonymous memory aligned
// to the huge-page size, advises the kernel to back it with huge pages, touches it, asks
// the kernel to collapse whatever the first touch left in small pages (a host whose free
// memory is fragmented grants only part of a large buffer in huge pages at fault time;
// such buffers measured 4-15 GB/s after kernel runs), and registers it with CUDA; where
// huge pages are unavailable it is ordinary registered memory.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>
#include <sys/mman.h>
#include <unistd.h>

#include <map>
#include <mutex>

#include "gk_internal.cuh"

namespace {

struct Mapping {
  void *base;
  size_t len;
};

std::mutex g_host_mu;
std::map<void *, Mapping> g_host_maps;

size_t huge_page_bytes() {
  size_t hp = 0;
  FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r");
  if (f) {
    unsigned long long v = 0;
    if (fscanf(f, "%llu", &v) == 1) hp = (size_t)v;
    fclose(f);
  }
  const size_t pg = (size_t)sysconf(_SC_PAGESIZE);
  if (hp < pg || (hp & (hp - 1)) != 0) hp = pg;
  return hp;
}

}  // namespace

extern "C" int gk_host_alloc(size_t bytes, void **ptr) {
  if (!ptr || bytes == 0) return GK_INVALID_ARG;
  *ptr = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return GK_NO_DEVICE;
  }
  const size_t hp = huge_page_bytes();
  const size_t len = (bytes + hp - 1) / hp * hp;
  const size_t span = len + hp;  // room to align the start to a huge page
  void *raw = mmap(nullptr, span, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return GK_OUT_OF_MEMORY;
  char *start = (char *)(((uintptr_t)raw + hp - 1) / hp * hp);
  // give back the unaligned head and the unused tail
  if (start > (char *)raw) munmap(raw, (size_t)(start - (char *)raw));
  char *end = start + len;
  if ((char *)raw + span > end) munmap(end, (size_t)((char *)raw + span - end));
#ifdef MADV_HUGEPAGE
  madvise(start, len, MADV_HUGEPAGE);
#endif
  memset(start, 0, len);  // populate now (huge pages where the kernel grants them)
#ifndef MADV_COLLAPSE
#define MADV_COLLAPSE 25
#endif
  // best effort (Linux 6.1 and later): synchronous collapse of the range into huge pages;
  // an older kernel or a failed compaction leaves the small pages, which still work
  if (hp > (size_t)sysconf(_SC_PAGESIZE)) madvise(start, len, MADV_COLLAPSE);
  if (cudaHostRegister(start, len, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(start, len);
    return GK_CUDA_ERROR;
  }
  {
    std::lock_guard<std::mutex> lock(g_host_mu);
    g_host_maps[start] = Mapping{start, len};
  }
  *ptr = start;
  return GK_OK;
}

extern "C" int gk_host_free(void *ptr) {
  Mapping mp;
  {
    std::lock_guard<std::mutex> lock(g_host_mu);
    auto it = g_host_maps.find(ptr);
    if (it == g_host_maps.end()) return GK_INVALID_ARG;
    mp = it->second;
    g_host_maps.erase(it);
  }
  int rc = GK_OK;
  if (cudaHostUnregister(mp.base) != cudaSuccess) {
    cudaGetLastError();
    rc = GK_CUDA_ERROR;
  }
  munmap(mp.base, mp.len);
  return rc;
}
