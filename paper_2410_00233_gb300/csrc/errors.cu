// Thread-local error messages of the C ABI.
#include <stdarg.h>
#include <stdio.h>

#include "kpsb_internal.cuh"

namespace kpsb {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

}  // namespace kpsb

extern "C" const char* kpsb_last_error(void) { return kpsb::g_err; }
