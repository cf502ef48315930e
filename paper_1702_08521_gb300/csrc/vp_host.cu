// vp_host.cu -- page-locked host buffers on transparent huge pages for the
// host <-> device copies of f (see vp_host_alloc in vlasov.h).
#include <sys/mman.h>
#include <unistd.h>

#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "vp_internal.cuh"

namespace {

struct Mapping {
    void *base;  // what mmap returned
    size_t len;  // its length
};

std::mutex g_host_mu;
std::unordered_map<void *, Mapping> g_host_maps;

// the kernel's transparent huge-page size (2 MB where it cannot be read)
size_t huge_page_size() {
    size_t hp = 2u << 20;
    if (FILE *fh = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (std::fscanf(fh, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) hp = (size_t)v;
        std::fclose(fh);
    }
    return hp;
}

}  // namespace

extern "C" {

int vp_host_alloc(size_t bytes, void **out) {
    if (!out || bytes == 0) return VP_EINVAL;
    *out = nullptr;
    const size_t hp = huge_page_size();
    const size_t len = (bytes + hp - 1) / hp * hp;
    // one huge page of slack so that the buffer can start on a huge-page boundary
    void *base = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (base == MAP_FAILED) return VP_ENOMEM;
    const uintptr_t b = reinterpret_cast<uintptr_t>(base);
    void *p = reinterpret_cast<void *>((b + hp - 1) / hp * hp);
    madvise(p, len, MADV_HUGEPAGE);  // advice only: base pages where the kernel has no huge ones
    if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(base, len + hp);
        return VP_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        g_host_maps[p] = Mapping{base, len + hp};
    }
    *out = p;
    return VP_OK;
}

int vp_host_free(void *p) {
    Mapping m;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_maps.find(p);
        if (it == g_host_maps.end()) return VP_EINVAL;
        m = it->second;
        g_host_maps.erase(it);
    }
    const cudaError_t e = cudaHostUnregister(p);
    munmap(m.base, m.len);
    return e == cudaSuccess ? VP_OK : VP_ECUDA;
}

}  // extern "C"
