// Shared host-side helpers of the C ABI: status handling and the per-thread error text.
#pragma once
#include <cuda_runtime.h>

#include <cstdio>
#include <exception>
#include <new>
#include <stdexcept>
#include <string>

#include "../../include/yateto_gb300.h"

namespace yt {

void set_last_error(const std::string& msg);
void clear_last_error();

// Thrown inside the library, converted to a status at the ABI boundary.
struct Error : std::runtime_error {
  yt_status status;
  Error(yt_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

inline void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of the runtime
    throw Error(e == cudaErrorMemoryAllocation ? YT_ERR_OOM : YT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  }
}

// Runs `f`, mapping exceptions to a yt_status and recording the message.
template <typename F>
yt_status guarded(F&& f) {
  try {
    clear_last_error();
    f();
    return YT_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return YT_ERR_OOM;
  } catch (const std::invalid_argument& e) {
    set_last_error(e.what());
    return YT_ERR_INVALID;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return YT_ERR_INVALID;
  }
}

#define YT_REQUIRE(cond, status, msg)            \
  do {                                           \
    if (!(cond)) throw ::yt::Error(status, msg); \
  } while (0)

}  // namespace yt
