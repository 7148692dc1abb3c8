// Host worker pool of parallel_for (hostpool.h).
#include "hostpool.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace dgasm {

namespace {

struct Job {
  const std::function<void(int)>* fn = nullptr;
  int n = 0;
  std::atomic<int> next{0};   // next index to hand out
  std::atomic<int> done{0};   // indices finished
  std::mutex mu;
  std::condition_variable cv;
};

thread_local bool t_in_job = false;

class Pool {
 public:
  static Pool& get() {
    static Pool pool;
    return pool;
  }
  int width() const { return (int)workers_.size() + 1; }

  void run(int n, const std::function<void(int)>& fn) {
    if (n <= 0) return;
    if (workers_.empty() || n == 1 || t_in_job) {
      for (int i = 0; i < n; ++i) fn(i);
      return;
    }
    auto job = std::make_shared<Job>();
    job->fn = &fn;
    job->n = n;
    {
      std::lock_guard<std::mutex> lk(mu_);
      queue_.push_back(job);
    }
    cv_.notify_all();
    work(*job);   // the caller takes indices too (so a job always finishes, even with no worker awake)
    std::unique_lock<std::mutex> lk(job->mu);
    job->cv.wait(lk, [&] { return job->done.load() == n; });
  }

 private:
  Pool() {
    const unsigned hc = std::thread::hardware_concurrency();
    const int nw = (int)std::min(15u, hc > 1 ? hc - 1 : 0u);
    for (int i = 0; i < nw; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }

  static void work(Job& job) {
    const bool prev = t_in_job;
    t_in_job = true;
    for (int i = job.next.fetch_add(1); i < job.n; i = job.next.fetch_add(1)) {
      (*job.fn)(i);
      if (job.done.fetch_add(1) + 1 == job.n) {
        std::lock_guard<std::mutex> lk(job.mu);
        job.cv.notify_all();
      }
    }
    t_in_job = prev;
  }

  void loop() {
    for (;;) {
      std::shared_ptr<Job> job;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || !queue_.empty(); });
        if (stop_) return;
        job = queue_.front();
        if (job->next.load() >= job->n) {   // every index handed out: the job leaves the queue
          queue_.pop_front();
          continue;
        }
      }
      work(*job);
    }
  }

  std::vector<std::thread> workers_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::shared_ptr<Job>> queue_;
  bool stop_ = false;
};

}  // namespace

void parallel_for(int n, const std::function<void(int)>& fn) { Pool::get().run(n, fn); }

int pool_width() { return Pool::get().width(); }

}  // namespace dgasm
