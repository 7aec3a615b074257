// Shared state of the device doubles (device_doubles.cpp) and the scenario
// runner (scenario.cpp) of the host-planning test.  Test infrastructure only.
#pragma once

#include <cstddef>
#include <cstdint>

namespace hp {
struct Checks {
  long long failures = 0;
  long long gemm_launches = 0, gemm_tiles = 0;        // FP64 FMA products (factor and traversal)
  long long emu_launches = 0, emu_tiles = 0, emu_splits = 0;
  long long tc_launches = 0, tc_tiles = 0;            // the precision form's TF32 products
  long long copy_launches = 0, copy_tasks = 0;
  long long other_launches = 0;
};
extern int rank_value;          // what a rank read back from the "device" holds
extern Checks checks;
extern uint64_t digest;         // FNV-1a of every checked task array, in launch order
}  // namespace hp
