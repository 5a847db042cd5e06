// The process-wide device lock's type (plain C++, no CUDA: the host tests compile it alone).
#pragma once

#include <condition_variable>
#include <mutex>

namespace iga {

// A reader-writer lock that admits a waiting writer before new readers.  std::shared_mutex
// (glibc's rwlock) prefers readers: with several setup threads whose eigensolves overlapped,
// a graph capture or the autotuner waited for a moment with no reader at all (up to 0.2 s).
class DeviceLock {
 public:
  void lock() {
    std::unique_lock<std::mutex> lk(m_);
    ++waiting_writers_;
    cv_.wait(lk, [&] { return !writer_ && readers_ == 0; });
    --waiting_writers_;
    writer_ = true;
  }
  void unlock() {
    {
      std::lock_guard<std::mutex> lk(m_);
      writer_ = false;
    }
    cv_.notify_all();
  }
  void lock_shared() {
    std::unique_lock<std::mutex> lk(m_);
    cv_.wait(lk, [&] { return !writer_ && waiting_writers_ == 0; });
    ++readers_;
  }
  void unlock_shared() {
    bool last;
    {
      std::lock_guard<std::mutex> lk(m_);
      last = --readers_ == 0;
    }
    if (last) cv_.notify_all();
  }

 private:
  std::mutex m_;
  std::condition_variable cv_;
  int readers_ = 0, waiting_writers_ = 0;
  bool writer_ = false;
};

}  // namespace iga
