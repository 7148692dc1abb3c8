// A process-wide pool of host worker threads for the data-parallel loops of the host plan (partitions, orderings,
// the permuted matrix, envelopes).  Creating threads for every loop of every setup cost more than some loops
// themselves; the pool's threads are created once and sleep between jobs.
#pragma once

#include <functional>

namespace dgasm {

// Runs fn(i) for every i in [0, n) on the pool's threads and the calling thread, and returns when all have
// run.  Indices are handed out one at a time in ascending order, so results are deterministic whenever fn(i)
// writes only its own outputs.  Safe to call from several threads at once, and from inside fn (a nested call
// runs its loop on the calling thread alone).
void parallel_for(int n, const std::function<void(int)>& fn);

// Worker threads of the pool plus the caller (1 when the host has a single core).
int pool_width();

}  // namespace dgasm
