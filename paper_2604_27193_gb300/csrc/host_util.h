// host_util.h -- thread-local error reporting for the C ABI.
#pragma once

#include <string>

#include "../../include/aeb.h"

namespace aeb {

void clear_error();
aeb_status fail(aeb_status code, const std::string &msg);

}  // namespace aeb
