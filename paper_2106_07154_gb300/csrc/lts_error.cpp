// lts_error.cpp -- thread-local last-error message of the C ABI.
#include "lts_error.h"

#include <cstdio>

#include "../../include/lts.h"

namespace lts {
namespace {
thread_local char g_msg[512] = "";
}

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

const char* last_error() { return g_msg; }
}  // namespace lts

extern "C" const char* lts_last_error(void) { return lts::last_error(); }
