// Adam's per-step prologue (Sec. 3.1: Adam with torch.optim.Adam semantics, plus
// dynamic loss scaling): one thread reads the flags the step's kernels raised and
// decides whether the pending update is applied or skipped, updates the loss
// scale and the step count, and computes the bias corrections the update reads.
// Shared by the optimizer's own prologue kernel and by the training step's loss
// kernel, which runs it right after the loss when an optimizer step follows.
#pragma once

#include <cuda_runtime.h>

#include "nh_internal.h"

namespace nh {

struct AdamHyper {
    float lr, beta1, beta2;
    int growth;   // growth interval of the dynamic loss scale; 0: fixed scale
};

__device__ __forceinline__ void adam_prologue(DeviceState* st, const AdamHyper& h) {
    const uint32_t flags = st->flags;
    const bool skip = (flags & NH_FLAG_NONFINITE) != 0u;
    st->flags = 0u;
    st->inv_scale = 1.f / st->loss_scale;
    if (skip) {
        st->skip = 1u;
        st->last_flags = flags | NH_FLAG_SKIPPED;
        if (h.growth > 0) {
            st->loss_scale = fmaxf(st->loss_scale * 0.5f, 1.f);
            st->good_steps = 0;
        }
        return;
    }
    st->skip = 0u;
    st->last_flags = flags;
    const int t = st->step + 1;
    st->step = t;
    st->step_size = h.lr / (1.f - powf(h.beta1, (float)t));
    st->inv_bc2_sqrt = 1.f / sqrtf(1.f - powf(h.beta2, (float)t));
    if (h.growth > 0) {
        if (++st->good_steps >= h.growth) {
            st->loss_scale = st->loss_scale * 2.f;
            st->good_steps = 0;
        }
    }
}

}  // namespace nh
