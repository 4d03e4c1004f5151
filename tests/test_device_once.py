"""Host logic of the once-per-device set-up of the kernel launchers (CPU).

Kernel attributes belong to a device context, so every launcher sets them
once per device (csrc/device_once.h).  This compiles a small C++ driver
against that header with the host compiler and checks, with 16 threads
racing on three device indices, that each device's set-up ran exactly once,
an unused device's never, and an out-of-range index's on every call.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2105_03297_gb300", "csrc")

DRIVER = r"""
#include "device_once.h"
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>
int main() {
  rve::DeviceOnce once;
  std::atomic<int> runs[4];
  for (auto& r : runs) r = 0;
  std::atomic<int> outside{0};
  std::vector<std::thread> th;
  for (int t = 0; t < 16; ++t)
    th.emplace_back([&, t] {
      for (int k = 0; k < 200; ++k) {
        const int d = (t + k) % 3;
        once.run(d, [&] { runs[d]++; });
      }
      once.run(-1, [&] { outside++; });
      once.run(rve::kMaxDevices, [&] { outside++; });
    });
  for (auto& x : th) x.join();
  std::printf("%d %d %d %d %d\n", runs[0].load(), runs[1].load(), runs[2].load(), runs[3].load(), outside.load());
  return 0;
}
"""


def test_setup_runs_once_per_device(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "once.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "once"
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert [int(v) for v in out] == [1, 1, 1, 0, 32]
