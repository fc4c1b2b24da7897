// The device-resident serving loop (oo_serve_start_resident): the layout
// shared by its host scheduler and its two persistent worker kernels.
//
// The host admits requests by free device memory and, per request, copies
// the inputs and a descriptor to the device and appends work entries to two
// rings in device memory; it then publishes them by raising a counter in
// mapped host memory.  No kernel is launched per request: the workers,
// launched once when serving starts, walk the rings:
//   - the SIMT ring (serve_resident.cu; 512-thread CTAs): digit splits of
//     FP64-equivalent GEMMs, FFT passes, Jacobi setup and stencil sweeps.  An entry has `nitems` items; CTA c takes items i with
//     (i + rot) % CTAs == c.  Every CTA reads every entry in order, so an
//     entry's dependency (an earlier entry) is always held by CTAs that are
//     running; items count into the entry's counter and the item that
//     completes it finishes the entry (the Jacobi residual sum, the request's
//     done flag);
//   - the tile ring (gemm_eq_group.cu; the grouped tensor-core kernel's
//     roles): one entry per output tile, tile t on CTA t % CTAs, which waits
//     for its GEMM's split entry before loading.
// Entry counters never reset: the host tracks every counter's running base.
// A request is done when the device writes its generation into done[slot]
// (mapped host memory); the host then copies the outputs back.  Every
// device wait is bounded (about one second); when idle the host publishes
// keep-alive entries so that waiting workers never reach the bound.
#pragma once

#include <cstdint>

namespace oo {
namespace res {

constexpr int kRingCap = 1 << 16;  // entries per ring
constexpr int kMaxCtas = 256;
constexpr int kSlots = 1024;       // request descriptors in flight
constexpr int kSlicePitch = 2048;  // BF16 row pitch of the digit-slice region (GEMM k <= 2048)
constexpr int kSimtThreads = 512;

enum EntryType {
    kNop = 0,
    kStop = 1,
    kSplit = 2,       // FP64-equivalent GEMM digit split: aux A-row items (16 rows), then B column items (64)
    // 3: unused (FFT scales come from the passes themselves)
    kFftWhole = 4,    // FFT of length <= 4096: one item
    kFftCols = 5,     // four-step column pass: item i = columns [i C, (i + 1) C)
    kFftRows = 6,     // four-step row pass
    kJacSetup = 7,    // Jacobi setup nests N0, N1: chunks of the padded grid (float4 units)
    kJacStencil = 8   // N2 for iteration aux (p and wrk2 alternate; see the item): chunks of column slabs
};

// control block in mapped pinned host memory
struct Ctl {
    volatile unsigned long long pub_simt;   // host: SIMT entries [0, pub_simt) are valid
    volatile unsigned long long pub_tiles;  // host: tile entries [0, pub_tiles) are valid
    volatile unsigned long long simt_progress[kMaxCtas];  // device: entries each SIMT CTA has passed
    volatile unsigned long long tile_progress[kMaxCtas];  // device: tile entries each tensor CTA has taken
    volatile unsigned done[kSlots];         // device: a request's generation once it is complete
    volatile unsigned fault;                // device: a bounded wait ran out (the workers stop)
    volatile unsigned alive[2 * kMaxCtas];  // device: 1 once each worker CTA runs (SIMT, then tensor)
    volatile unsigned long long stuck_at, stuck_seen;  // device: the entry a timed-out SIMT wait was for, and
                                                       // the publication count it last read
};

// SIMT ring entry (device memory)
struct Entry {
    int32_t type, slot, nitems, rot;
    uint32_t ctr, target;   // this entry's counter and the value that marks it complete
    int32_t dep_ctr;        // counter this entry waits for (-1: none) until it reaches dep_target
    uint32_t dep_target;
    int32_t aux;            // kSplit: A items; kJacStencil: iteration; FFT: log2 pass length
    uint32_t gen;           // written to done[slot] when a `last` entry completes
    int32_t last;
    int32_t pad;
};

// Jacobi request descriptor (device memory)
struct JacDesc {
    float *arr[14];  // a0..a3, b0..b2, c0..c2, bnd, wrk1, p, wrk2 (I x J x pitch floats each)
    double *res;     // iters
    double *partials;  // two sets (iteration parity) of one partial per stencil item
    int32_t I, J, K, pitch, iters;
    int32_t chunk, chunk4;  // stencil units (column x slab) per item; float4 units per setup item
    float omega;
    int32_t nseg;           // slabs of interior planes
};

}  // namespace res
}  // namespace oo
