// Planner: placeholder entry points (the Einstein-expression planner is added next).
#include "common.h"

struct yt_plan {};

extern "C" yt_status yt_plan_create(const char*, const yt_tensor_desc*, int32_t, yt_precision,
                                    yt_plan** out) {
  if (out) *out = nullptr;
  yt::set_last_error("planner not built");
  return YT_ERR_UNSUPPORTED;
}
extern "C" yt_status yt_plan_stats_get(const yt_plan*, yt_plan_stats*) { return YT_ERR_UNSUPPORTED; }
extern "C" yt_status yt_plan_eqspp(const yt_plan*, int32_t, int32_t, uint8_t*) { return YT_ERR_UNSUPPORTED; }
extern "C" yt_status yt_execute_batched(const yt_plan*, void* const*, int64_t, yt_stream) { return YT_ERR_UNSUPPORTED; }
extern "C" void yt_plan_destroy(yt_plan* p) { delete p; }
