// prof.cu -- optional per-context stage timing with CUDA events recorded on the
// stream each kernel is launched on (enabled by LSG_SETUP_PROFILE).  A solve
// records one event pair around every triangular-sweep kernel and every
// matrix-free product it launches; the totals are read after the solve has
// synchronised, so the timing adds no host synchronisation to the solve.
#include <vector>

#include "lsg_internal.cuh"

namespace lsg {

struct Prof {
    struct Rec {
        int stage, tag;
        cudaEvent_t e0, e1;
    };
    std::vector<Rec> recs;   // event pool, reused solve after solve
    size_t used = 0;
    int tag = -1;            // iteration tag of the records being made (-1: none)
    int next_tag = 0;
    std::vector<char> done;  // per tag: the iteration did its work
    double us[PROF_STAGES] = {};
    long long calls[PROF_STAGES] = {};
    long long dropped = 0;   // records beyond the pool cap (not timed)
};

constexpr size_t kProfCap = 1 << 14;

int prof_begin(lsg_ctx *c, int stage, cudaStream_t s, int *slot)
{
    *slot = -1;
    Prof *P = c->prof;
    if (!P) return LSG_OK;
    if (P->used == P->recs.size()) {
        if (P->recs.size() >= kProfCap) {
            ++P->dropped;
            return LSG_OK;
        }
        Prof::Rec r{stage, -1, nullptr, nullptr};
        LSG_CK(cudaEventCreate(&r.e0));
        LSG_CK(cudaEventCreate(&r.e1));
        P->recs.push_back(r);
    }
    Prof::Rec &r = P->recs[P->used];
    r.stage = stage;
    r.tag = P->tag;
    LSG_CK(cudaEventRecord(r.e0, s));
    *slot = (int)P->used++;
    return LSG_OK;
}

int prof_end(lsg_ctx *c, int slot, cudaStream_t s)
{
    if (slot < 0 || !c->prof) return LSG_OK;
    LSG_CK(cudaEventRecord(c->prof->recs[slot].e1, s));
    return LSG_OK;
}

void prof_reset(lsg_ctx *c)
{
    Prof *P = c->prof;
    if (!P) return;
    P->used = 0;
    P->dropped = 0;
    P->tag = -1;
    P->next_tag = 0;
    P->done.clear();
    for (int i = 0; i < PROF_STAGES; ++i) P->us[i] = 0.0, P->calls[i] = 0;
}

// A fresh tag for the next iteration the caller queues (also without the profiler,
// so that callers can count queued iterations the same way).
int prof_tag(lsg_ctx *c)
{
    Prof *P = c->prof;
    return P ? P->next_tag++ : 0;
}

void prof_set_tag(lsg_ctx *c, int tag)
{
    if (c->prof) c->prof->tag = tag;
}

void prof_mark_done(lsg_ctx *c, int first_tag, int count)
{
    Prof *P = c->prof;
    if (!P || count <= 0) return;
    if ((int)P->done.size() < first_tag + count) P->done.resize(first_tag + count, 0);
    for (int t = first_tag; t < first_tag + count; ++t) P->done[t] = 1;
}

// Sum the recorded pairs into the stage totals (the events must have completed).
int prof_collect(lsg_ctx *c)
{
    Prof *P = c->prof;
    if (!P) return LSG_OK;
    for (size_t i = 0; i < P->used; ++i) {
        float ms = 0.0f;
        const int tag = P->recs[i].tag;
        if (tag >= 0 && (tag >= (int)P->done.size() || !P->done[tag])) continue;  // queued after the stop
        LSG_CK(cudaEventSynchronize(P->recs[i].e1));
        LSG_CK(cudaEventElapsedTime(&ms, P->recs[i].e0, P->recs[i].e1));
        P->us[P->recs[i].stage] += 1000.0 * ms;
        P->calls[P->recs[i].stage] += 1;
    }
    P->used = 0;
    P->tag = -1;
    return LSG_OK;
}

void prof_create(lsg_ctx *c) { c->prof = new Prof(); }

void prof_destroy(lsg_ctx *c)
{
    Prof *P = c->prof;
    if (!P) return;
    for (auto &r : P->recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    delete P;
    c->prof = nullptr;
}

long long prof_query(const lsg_ctx *c, int stage, bool calls)
{
    const Prof *P = c->prof;
    if (!P || stage < 0 || stage >= PROF_STAGES) return -1;
    return calls ? P->calls[stage] : (long long)(P->us[stage] + 0.5);
}

}  // namespace lsg
