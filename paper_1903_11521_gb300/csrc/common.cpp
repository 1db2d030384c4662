// Status strings, per-thread error text, version.
#include "common.h"

namespace yt {
namespace {
thread_local std::string g_last_error;
}
void set_last_error(const std::string& msg) { g_last_error = msg; }
void clear_last_error() { g_last_error.clear(); }
}  // namespace yt

extern "C" const char* yt_status_string(yt_status s) {
  switch (s) {
    case YT_OK: return "YT_OK";
    case YT_ERR_INVALID: return "YT_ERR_INVALID: invalid argument";
    case YT_ERR_PARSE: return "YT_ERR_PARSE: malformed expression";
    case YT_ERR_SHAPE: return "YT_ERR_SHAPE: inconsistent shapes";
    case YT_ERR_UNSUPPORTED: return "YT_ERR_UNSUPPORTED: no kernel for this request";
    case YT_ERR_OOM: return "YT_ERR_OOM: out of memory";
    case YT_ERR_CUDA: return "YT_ERR_CUDA: CUDA runtime error";
    case YT_ERR_TIMEOUT: return "YT_ERR_TIMEOUT: bounded device wait ran out";
  }
  return "unknown yt_status";
}

extern "C" const char* yt_last_error(void) { return yt::g_last_error.c_str(); }

extern "C" const char* yt_version(void) { return "yateto_gb300 0.1 sm_103a"; }
