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
// Where a caller's pointer lives: 0 host memory (pageable or page-locked),
// 1 device memory of `device` or managed memory, 2 device memory of another
// GPU (which kernels on `device` must not be given).
int pointer_kind(const void *p, int device);
}  // namespace bang
