// Host-side helpers shared by the C-ABI entry points: error recording and
// workspace carving.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>

#include "tv.h"

namespace tvh {

void set_error(const char *fmt, ...);
void clear_error();

// Returns TV_ERR_CUDA (with a message) if e is an error, else TV_OK.
tv_status check_cuda(cudaError_t e, const char *what);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over a caller-provided workspace (256-byte aligned slices).
struct Carver {
    char *base;
    size_t used;
    explicit Carver(void *b) : base(static_cast<char *>(b)), used(0) {}
    template <class T>
    T *take(size_t count)
    {
        used = align_up(used, 256);
        T *p = base ? reinterpret_cast<T *>(base + used) : nullptr;
        used += sizeof(T) * count;
        return p;
    }
};

// Launch shape for a batch of `warps` warps, one chain per lane.
struct Shape {
    int wpb;
    long long blocks;
};
Shape batch_shape(long long warps, int sm_count);
int sm_count_current();

}  // namespace tvh
