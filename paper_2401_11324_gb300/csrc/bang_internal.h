// Internal helpers shared by the library's translation units (not part of the C ABI).
#pragma once

#include <string>

namespace bang {
// Record the message returned by bang_last_error() for the calling thread.
void set_error(const std::string &msg);
}  // namespace bang
