"""Host check of the process-wide device lock (csrc/device_lock.h): setup threads take it
shared around cuSOLVER eigensolves and exclusively around graph captures, the tensor-core
autotuner and kernel attribute changes.  A waiting writer must get in before readers that
arrive after it (with a reader-preferring lock a short capture waited behind overlapping
eigensolves), and mixed traffic from many threads must always finish.  Compiled with g++."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_04384_gb300", "csrc")

PROG = r"""
#include <atomic>
#include <chrono>
#include <cstdio>
#include <random>
#include <shared_mutex>
#include <thread>
#include <vector>
#include "device_lock.h"
using namespace std::chrono_literals;
int main() {
  iga::DeviceLock L;
  // order: reader 1 holds the lock; the writer asks; reader 2 asks after the writer
  std::atomic<int> seq{0};
  int r1 = -1, w = -1, r2 = -1;
  std::thread t1([&] { std::shared_lock<iga::DeviceLock> g(L); r1 = seq++; std::this_thread::sleep_for(200ms); });
  std::this_thread::sleep_for(30ms);
  std::thread tw([&] { std::unique_lock<iga::DeviceLock> g(L); w = seq++; std::this_thread::sleep_for(20ms); });
  std::this_thread::sleep_for(30ms);
  std::thread t2([&] { std::shared_lock<iga::DeviceLock> g(L); r2 = seq++; });
  t1.join(); tw.join(); t2.join();
  // mixed traffic: readers may overlap, a writer is alone
  std::atomic<int> readers{0}, writers{0}, bad{0};
  std::vector<std::thread> th;
  for (int i = 0; i < 12; ++i)
    th.emplace_back([&, i] {
      std::mt19937 g(i);
      for (int k = 0; k < 400; ++k) {
        if (g() % 4 == 0) {
          std::unique_lock<iga::DeviceLock> lk(L);
          if (writers++ != 0 || readers != 0) ++bad;
          std::this_thread::sleep_for(std::chrono::microseconds(g() % 50));
          --writers;
        } else {
          std::shared_lock<iga::DeviceLock> lk(L);
          ++readers;
          if (writers != 0) ++bad;
          std::this_thread::sleep_for(std::chrono::microseconds(g() % 50));
          --readers;
        }
      }
    });
  for (auto &t : th) t.join();
  std::printf("%d %d %d %d\n", r1, w, r2, bad.load());
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_device_lock_prefers_waiting_writer_and_excludes(tmp_path):
    src = tmp_path / "l.cpp"
    src.write_text(PROG)
    exe = tmp_path / "l"
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    r1, w, r2, bad = map(int, r.stdout.split())
    assert (r1, w, r2) == (0, 1, 2), r.stdout  # the writer before the later reader
    assert bad == 0, r.stdout
