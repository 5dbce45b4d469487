// ScratchScope: the stream-ordered scratch buffers of one library call.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace ptrom {

// The stream-ordered scratch buffers of one call: release() hands them back
// on the normal path; on an early error return the destructor does, so no
// return path leaks device memory.
struct ScratchScope {
    cudaStream_t st;
    std::vector<void *> bufs;
    explicit ScratchScope(cudaStream_t s) : st(s) {}
    ScratchScope(const ScratchScope &) = delete;
    ScratchScope &operator=(const ScratchScope &) = delete;
    template <typename T> int alloc(T **p, size_t bytes) {
        void *q = nullptr;
        const int e = scratch_alloc(&q, bytes, st);
        if (e == PTROM_OK) {
            bufs.push_back(q);
            *p = (T *)q;
        }
        return e;
    }
    int release() {
        int first = PTROM_OK;
        for (void *q : bufs) {
            const int e = scratch_free(q, st);
            if (first == PTROM_OK) first = e;
        }
        bufs.clear();
        return first;
    }
    ~ScratchScope() {
        for (void *q : bufs) cudaFreeAsync(q, st);
    }
};

}  // namespace ptrom
