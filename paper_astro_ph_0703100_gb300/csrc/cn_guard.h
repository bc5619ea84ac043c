// The C ABI boundary: no C++ exception leaves the library. Every entry point
// runs its body through guard(): host memory exhausted inside the library
// (std::bad_alloc from a plan's tables, the tuning map, a message string) or
// any other C++ runtime error becomes the status CN_ERR_HOST, with its
// message for cn_last_error_message, and the caller's state is as before
// the call failed.
#pragma once

#include <new>

#include "cunbody.h"

namespace cn {

// records msg as the last error without allocating if that fails (cn_api.cu)
cn_status fail_nothrow(cn_status st, const char* msg) noexcept;

template <class F>
cn_status guard(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail_nothrow(CN_ERR_HOST, "host memory allocation failed inside the library");
  } catch (...) {
    return fail_nothrow(CN_ERR_HOST, "a host-side C++ runtime error inside the library");
  }
}

// the same for entry points that return a value (on_error when anything was thrown)
template <class T, class F>
T guard_value(T on_error, F&& body) noexcept {
  try {
    return body();
  } catch (...) {
    return on_error;
  }
}

}  // namespace cn
