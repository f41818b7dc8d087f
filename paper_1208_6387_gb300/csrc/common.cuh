// Shared host/device utilities of the fetirp library (no method arithmetic here).
#pragma once
#include <cstdlib>

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

namespace fetirp {

// Error carried from deep inside the library to the C ABI boundary, where it becomes a status code.
struct Error : public std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define FETIRP_CUDA(call)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      throw ::fetirp::Error(e_ == cudaErrorMemoryAllocation ? 2 : 5,                            \
                            std::string(#call) + ": " + cudaGetErrorString(e_) + " at " +       \
                                __FILE__ + ":" + std::to_string(__LINE__));                     \
  } while (0)

// Every kernel launch of the library is followed by this check, which also counts the launch (per host
// thread: a context is driven by one thread at a time, so its counts stay exact when several run at once).
extern thread_local unsigned long long g_launch_count;
#define FETIRP_LAUNCH_CHECK()        \
  do {                               \
    ++::fetirp::g_launch_count;      \
    FETIRP_CUDA(cudaGetLastError()); \
  } while (0)

// Owning device buffer (cudaMalloc / cudaFree).
inline bool poison_allocations() {
  static const bool on = [] {
    const char* v = std::getenv("FETIRP_POISON");
    return v && v[0] == '1';
  }();
  return on;
}

// Caller-supplied device allocator (fetirp_options.alloc / free).  Every entry point of the library installs
// its context's hooks for the calling host thread while it runs; with no hooks installed device buffers come
// from cudaMalloc.  A buffer remembers the free hook it was allocated with.
typedef void* (*DevAllocFn)(size_t bytes, void* stream, void* user);
typedef void (*DevFreeFn)(void* ptr, void* user);
struct DevAllocator {
  DevAllocFn alloc = nullptr;
  DevFreeFn free = nullptr;
  void* user = nullptr;
  void* stream = nullptr;
};
inline DevAllocator& current_allocator() {
  thread_local DevAllocator a;
  return a;
}
struct AllocatorScope {
  DevAllocator saved;
  explicit AllocatorScope(const DevAllocator& a) : saved(current_allocator()) { current_allocator() = a; }
  ~AllocatorScope() { current_allocator() = saved; }
  AllocatorScope(const AllocatorScope&) = delete;
  AllocatorScope& operator=(const AllocatorScope&) = delete;
};

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DevFreeFn free_fn = nullptr;   // set when the buffer came from a caller hook
  void* free_user = nullptr;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), free_fn(o.free_fn), free_user(o.free_user) {
    o.p = nullptr; o.n = 0; o.free_fn = nullptr; o.free_user = nullptr;
  }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; free_fn = o.free_fn; free_user = o.free_user;
      o.p = nullptr; o.n = 0; o.free_fn = nullptr; o.free_user = nullptr;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    const DevAllocator& a = current_allocator();
    if (a.alloc) {
      void* q = a.alloc(count * sizeof(T), a.stream, a.user);
      if (!q) throw Error(2, "the caller's device allocator returned NULL for " + std::to_string(count * sizeof(T)) +
                                 " bytes");
      if (reinterpret_cast<uintptr_t>(q) & 255) {
        a.free(q, a.user);
        throw Error(1, "the caller's device allocator returned a pointer that is not 256-byte aligned");
      }
      p = static_cast<T*>(q);
      free_fn = a.free;
      free_user = a.user;
    } else {
      FETIRP_CUDA(cudaMalloc(&p, count * sizeof(T)));
    }
    // FETIRP_POISON=1 (debugging and tests): fill every new allocation with NaN bytes so that a read of memory
    // the library never wrote shows up as NaN in the results; synchronous, so no stream work overtakes it
    if (poison_allocations()) {
      FETIRP_CUDA(cudaMemset(p, 0xFF, count * sizeof(T)));
      FETIRP_CUDA(cudaDeviceSynchronize());
    }
    n = count;
  }
  // grow-only reallocation (contents not kept)
  void ensure(size_t count) { if (count > n) alloc(count); }
  void release() {
    if (p) {
      if (free_fn) {
        // work on any of the library's streams may still read the buffer: finish it before the caller's
        // allocator can hand the memory out again (cudaFree synchronises the same way)
        cudaDeviceSynchronize();
        free_fn(p, free_user);
      } else {
        cudaFree(p);
      }
    }
    p = nullptr;
    n = 0;
    free_fn = nullptr;
    free_user = nullptr;
  }
  void upload(const T* h, size_t count, cudaStream_t s) {
    ensure(count);
    if (count) FETIRP_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void upload(const std::vector<T>& h, cudaStream_t s) { upload(h.data(), h.size(), s); }
  void zero(cudaStream_t s) { if (n) FETIRP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
inline long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

}  // namespace fetirp
