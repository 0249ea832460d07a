// Plain structures shared by the kernels and the host runtimes: the batch
// and serving-slot descriptors and the serving control block.  No CUDA types.
#pragma once

namespace stev {

// Control block of a serving kernel (device memory).  The host publishes a
// request by copying, in this order on one stream, its slot, then pub_seq,
// then published; kernels claim ids below `published` with compare-and-swap
// on `claim`.  `stop` != 0 makes warps stop claiming and leave once idle.
// `dropped` counts cells whose slot lookup gave an index outside the
// request (never expected; the cell is skipped instead of read).
// The kernel leaves as a whole: a warp idle for idle_ns counts itself in
// `idle_warps` (and out again when work appears); the warp that sees every
// warp counted sets `exiting`, after which nobody claims and every warp
// leaves once its cells are done.  The host zeroes both before a launch.
struct ServeCtl {
  unsigned long long claim;      // next unclaimed cell id
  unsigned long long published;  // ids below this are ready
  long long pub_seq;             // sequence number of the newest published request
  int stop;
  int dropped;
  int idle_warps;
  int exiting;
};

// Serving slot key: first cell id and sequence number in one 64-bit word,
// so that a reader racing with the host's rewrite of a retired slot sees
// either the old or the new pair, never a mix.
constexpr int kServeSeqBits = 20;  // sequence numbers are compared mod 2^20
constexpr unsigned long long kServeSeqMask = (1ULL << kServeSeqBits) - 1;
constexpr unsigned long long kServeMaxIds = 1ULL << (64 - kServeSeqBits);  // cell ids per server

// One independent batch of cells in a batched launch (its own arrays, size
// and fluid time step).  Layouts as for the single-batch entry points.
struct BatchDesc {
  const double* T;
  const double* P;
  const double* Y;        // [n][S]
  double* T_out;
  double* Y_out;          // [n][S]
  int* iters;
  unsigned char* status;
  double dt;
  long long n;
};

// One request slot of a serving kernel: the request's arrays (solved in
// place), its key (first cell id << kServeSeqBits | seq mod 2^kServeSeqBits;
// slot index = seq mod queue length) and its finished-cell count.
struct ServeSlot {
  BatchDesc d;
  unsigned long long key;
  unsigned long long done;
};

}  // namespace stev
