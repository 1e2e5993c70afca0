// Pinned host buffers for host-resident state (flb_host_alloc / flb_host_free).
//
// A box whose state lives in host memory crosses the host link twice per step
// (flb_box_step_host).  The copy engines reach the link's rate only from
// page-locked memory, and the rate they keep also depends on how the pages are
// mapped: memory that is taken as transparent huge pages, faulted in once and
// then registered with the driver streams at the same rate from the first call
// on, while small-page pinned memory showed slow first calls and stalls.  So
// the buffer is an anonymous mapping aligned to the huge-page size, advised to
// use huge pages, touched page by page (which also zeroes it) and registered.
#include <cuda_runtime.h>

#include <sys/mman.h>
#include <unistd.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>

#include "flb.h"

namespace {

struct Mapping {
    void *base;
    size_t len;
};

std::mutex g_mu;
std::map<uintptr_t, Mapping> g_maps;   // user pointer -> whole mapping

size_t huge_page_size()
{
    size_t hp = 0;
    if (FILE *f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (std::fscanf(f, "%llu", &v) == 1) hp = (size_t)v;
        std::fclose(f);
    }
    return hp;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

int flb_host_alloc(size_t nbytes, void **out)
{
    if (!out || nbytes == 0) return FLB_EINVAL;
    *out = nullptr;
    const long ps = sysconf(_SC_PAGESIZE);
    const size_t page = ps > 0 ? (size_t)ps : 4096;
    const size_t hp = huge_page_size();
    // huge-page alignment only where the buffer spans at least one huge page
    const size_t align = (hp > page && nbytes >= hp) ? hp : page;
    const size_t len = round_up(nbytes, page);
    const size_t span = len + (align > page ? align : 0);
    void *raw = mmap(nullptr, span, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == MAP_FAILED) return FLB_ENOMEM;
    char *p = static_cast<char *>(raw);
    if (align > page) {
        // keep only the aligned window of the over-sized mapping
        char *a = reinterpret_cast<char *>(round_up(reinterpret_cast<uintptr_t>(p), align));
        if (a > p) munmap(p, (size_t)(a - p));
        const size_t tail = (size_t)(p + span - (a + len));
        if (tail) munmap(a + len, tail);
        p = a;
        madvise(p, len, MADV_HUGEPAGE);   // advisory: without it the buffer is still correct
    }
    volatile char *v = p;
    for (size_t off = 0; off < len; off += page) v[off] = 0;
    if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(p, len);
        return FLB_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_maps[reinterpret_cast<uintptr_t>(p)] = Mapping{p, len};
    }
    *out = p;
    return FLB_OK;
}

int flb_host_free(void *ptr)
{
    if (!ptr) return FLB_OK;
    Mapping m;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_maps.find(reinterpret_cast<uintptr_t>(ptr));
        if (it == g_maps.end()) return FLB_EINVAL;
        m = it->second;
        g_maps.erase(it);
    }
    const cudaError_t e = cudaHostUnregister(m.base);
    munmap(m.base, m.len);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FLB_ECUDA;
    }
    return FLB_OK;
}

}  // extern "C"
