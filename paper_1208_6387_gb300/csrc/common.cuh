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

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    FETIRP_CUDA(cudaMalloc(&p, count * sizeof(T)));
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
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
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
