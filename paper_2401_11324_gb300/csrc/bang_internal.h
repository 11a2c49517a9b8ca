// Internal helpers shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>

struct bang_index;

namespace bang {
// Record the message returned by bang_last_error() for the calling thread.
void set_error(const std::string &msg);
// CUDA device and placement flags of an index.
int index_device(const bang_index *ix);
uint32_t index_placement(const bang_index *ix);
}  // namespace bang
