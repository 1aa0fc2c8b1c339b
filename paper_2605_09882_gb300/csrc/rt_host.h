// Host-side helpers shared by the library's translation units.
#pragma once

#include <string.h>

#include <algorithm>

#include "rt_internal.h"

namespace rt {
int set_error(int code, const char* msg);
int cuda_error(const char* where);
void clear_error();
}  // namespace rt
