// Once-per-device set-up for kernel launchers.
//
// Function attributes (the dynamic shared-memory limit, the carveout) belong
// to a device context: a kernel launched on a second device needs them set
// there again.  DeviceOnce runs a set-up function once per device index, and
// std::call_once makes the first run race-free when several host threads (the
// size groups of a batch solve) launch the same kernel together.  Host-only
// C++, no CUDA calls, so that its logic can be tested without a GPU.
#pragma once
#include <mutex>
#include <utility>

namespace rve {

constexpr int kMaxDevices = 64;

class DeviceOnce {
 public:
  // Runs fn the first time it is called for `device`; later calls for the same
  // device return at once (after the first call has finished).  A device
  // index outside [0, kMaxDevices) runs fn every time.
  template <class Fn> void run(int device, Fn&& fn) {
    if (device < 0 || device >= kMaxDevices) {
      fn();
      return;
    }
    std::call_once(flags_[device], std::forward<Fn>(fn));
  }

 private:
  std::once_flag flags_[kMaxDevices];
};

}  // namespace rve
