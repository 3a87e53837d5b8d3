// lts_error.h -- thread-local error message shared by the translation units
// of liblts.so (host code only).
#pragma once
#include <cstdarg>

namespace lts {
// Formats a message into the calling thread's error slot and returns `code`.
int set_error(int code, const char* fmt, ...);
const char* last_error();
}  // namespace lts
