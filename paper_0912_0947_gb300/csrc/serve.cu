// serve.cu -- continuous-batching request server over the batched kernels.
//
// Requests (embed or extract, one cover each, mixed sizes) are queued by
// stego_server_submit from any thread.  One dispatcher thread per server:
//   * polls the events of the batches in flight; a finished batch hands its
//     per-request results back as completions and releases its bytes from
//     the in-flight budget;
//   * whenever a slot (a CUDA stream with its own descriptor, result and
//     workspace buffers) is free, admits queued requests in arrival order
//     while their working-set bytes fit the budget, up to max_batch per
//     batch, and launches them as one batched embed and/or one batched
//     extract on that slot's stream.
// Stream-layout requests with k > 1 bits per byte or one carrying plane
// (which the batched kernels do not take) ride in the same batch as calls
// of their own to the single-cover entry points on the slot's stream; their
// results sit after the batched ones in the slot's result arrays.
// Requests that arrive while batches run are admitted into the next free
// slot as soon as the budget allows, so batches overlap on the device.  A
// request larger than the whole budget completes at once with
// STEGO_E_NOMEM instead of waiting forever.
//
// Device memory: the caller passes one arena (stego_server_arena_bytes) that
// holds every slot's descriptors, results and workspace; the server
// allocates no device memory.  Per slot it keeps pinned host copies of the
// descriptors and results (allocated once, at creation).
#ifdef __linux__
#include <sys/prctl.h>
#endif
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    stego_request req;
    double t_submit;
    uint64_t bytes;
};

struct Member {
    Pending p;
    bool embed;
    bool single;    // served by a single-cover call instead of the batched one
    uint32_t index; // into the slot's embed or extract arrays
    double t_dispatch;
};

// k > 1 bits per byte or one carrying plane in the stream layout.
bool single_cover_only(uint32_t flags)
{
    return (flags & STEGO_LAYOUT_MASK) == STEGO_LAYOUT_STREAM1 &&
           (flags & (STEGO_BITS_MASK | STEGO_PLANE_ONLY)) != 0;
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    stego_desc *h_desc_e = nullptr, *h_desc_x = nullptr;
    stego_result *h_res_e = nullptr, *h_res_x = nullptr;
    stego_desc *d_desc_e = nullptr, *d_desc_x = nullptr;
    stego_result *d_res_e = nullptr, *d_res_x = nullptr;
    void *d_ws_e = nullptr, *d_ws_x = nullptr;
    uint64_t ws_bytes = 0;
    std::vector<Member> members;
    bool busy = false;
    int launch_status = STEGO_OK;
};

uint64_t round256(uint64_t x) { return (x + 255u) & ~255ull; }

uint64_t slot_bytes(uint32_t max_batch)
{
    const uint64_t d = round256(sizeof(stego_desc) * (uint64_t)max_batch);
    const uint64_t r = round256(sizeof(stego_result) * (uint64_t)max_batch);
    const uint64_t w = round256(stego_batched_workspace_bytes(max_batch));
    return 2 * (d + r + w);
}

bool config_ok(const stego_server_config *c)
{
    return c && c->slots >= 1 && c->slots <= 16 && c->max_batch >= 1 && c->max_batch <= 8192 &&
           c->budget_bytes > 0 && stego::tune_ok(&c->tune_embed) && stego::tune_ok(&c->tune_extract);
}

// Working-set bytes of one request: what it reads and writes.
uint64_t request_bytes(const stego_request &r)
{
    if (r.op == STEGO_OP_EMBED)
        return 2 * r.cover_bytes + r.msg_bytes;
    return r.cover_bytes + r.msg_bytes;
}

} // namespace

struct stego_server {
    stego_server_config cfg;
    int device = 0;
    Clock::time_point t0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work; // dispatcher waits for submissions
    std::condition_variable cv_done; // clients wait for completions
    std::deque<Pending> queue;
    std::vector<stego_completion> done;
    uint64_t in_flight_bytes = 0;
    uint64_t peak_in_flight = 0; // largest in_flight_bytes seen
    uint64_t outstanding = 0;    // submitted, not yet completed
    uint64_t batches = 0;
    bool stop = false;
    double t_last_launch = -1.0; // dispatcher thread only
    std::thread th;

    double now() const
    {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }

    void complete_now(const Pending &p, int status, double t)
    {
        stego_completion c;
        std::memset(&c, 0, sizeof(c));
        c.tag = p.req.tag;
        c.status = status;
        c.t_submit = p.t_submit;
        c.t_dispatch = t;
        c.t_done = t;
        done.push_back(c);
        --outstanding;
    }

    // Finished batches -> completions.  Caller holds no lock.
    bool reap()
    {
        bool any = false;
        for (Slot &s : slots) {
            if (!s.busy)
                continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady)
                continue;
            const double t = now();
            const int err = (q == cudaSuccess && s.launch_status == STEGO_OK)
                                ? STEGO_OK
                                : (s.launch_status != STEGO_OK ? s.launch_status : STEGO_E_CUDA);
            if (q != cudaSuccess)
                cudaGetLastError();
            std::lock_guard<std::mutex> lk(mu);
            for (const Member &m : s.members) {
                const stego_result &r = m.embed ? s.h_res_e[m.index] : s.h_res_x[m.index];
                stego_completion c;
                std::memset(&c, 0, sizeof(c));
                c.tag = m.p.req.tag;
                c.changed = err == STEGO_OK ? r.changed : 0;
                c.sse = err == STEGO_OK ? r.sse : 0;
                c.msg_bytes = err == STEGO_OK ? r.msg_bytes : 0;
                c.status = err == STEGO_OK ? r.status : err;
                c.batch_size = (int32_t)s.members.size();
                c.t_submit = m.p.t_submit;
                c.t_dispatch = m.t_dispatch;
                c.t_done = t;
                done.push_back(c);
                in_flight_bytes -= m.p.bytes;
                --outstanding;
            }
            s.members.clear();
            s.busy = false;
            any = true;
        }
        if (any)
            cv_done.notify_all();
        return any;
    }

    // The slot's single-cover members of one direction, each a call of its
    // own on the slot's stream writing its result entry.  A request the call
    // refuses on the host gets that status in its result, as the batched
    // prep reports refused descriptors; only a CUDA failure fails the batch.
    int launch_singles(Slot &s, bool embed)
    {
        for (const Member &m : s.members) {
            if (!m.single || m.embed != embed)
                continue;
            const stego_request &r = m.p.req;
            const stego_geom *g = (r.flags & STEGO_PLANE_ONLY) ? &r.geom : nullptr;
            stego_result *res = (embed ? s.d_res_e : s.d_res_x) + m.index;
            const int st = embed ? stego_embed(r.cover, r.stego, r.cover_bytes, r.msg,
                                               r.msg_bytes, g, r.flags | STEGO_FUSE_STATS, res,
                                               s.stream)
                                 : stego_extract(r.cover, r.cover_bytes, r.msg, r.msg_bytes,
                                                 r.msg_len, g, r.flags, res, s.stream);
            if (st == STEGO_E_CUDA)
                return st;
            if (st != STEGO_OK && stego::write_result(res, 0, st, s.stream) != cudaSuccess)
                return STEGO_E_CUDA;
        }
        return STEGO_OK;
    }

    // Admit queued requests into a free slot and launch them.
    bool dispatch()
    {
        bool any = false;
        for (Slot &s : slots) {
            if (s.busy)
                continue;
            uint32_t ne = 0, nx = 0;
            {
                std::lock_guard<std::mutex> lk(mu);
                const double t = now();
                while (!queue.empty() && ne + nx < cfg.max_batch) {
                    Pending &p = queue.front();
                    if (p.req.op != STEGO_OP_EMBED && p.req.op != STEGO_OP_EXTRACT) {
                        complete_now(p, STEGO_E_INVAL, t);
                        queue.pop_front();
                        continue;
                    }
                    if (p.bytes > cfg.budget_bytes) {
                        complete_now(p, STEGO_E_NOMEM, t);
                        queue.pop_front();
                        continue;
                    }
                    if (in_flight_bytes + p.bytes > cfg.budget_bytes)
                        break; // arrival order: wait for the budget to free up
                    Member m;
                    m.p = p;
                    m.embed = p.req.op == STEGO_OP_EMBED;
                    m.single = single_cover_only(p.req.flags);
                    m.index = m.embed ? ne++ : nx++;
                    m.t_dispatch = t;
                    in_flight_bytes += p.bytes;
                    peak_in_flight = std::max(peak_in_flight, in_flight_bytes);
                    s.members.push_back(m);
                    queue.pop_front();
                }
                if (!done.empty())
                    cv_done.notify_all();
            }
            if (s.members.empty())
                break; // nothing admissible now
            stego::Trace trace_("stego_server batch");
            // batched members first (descriptors 0..nbe-1 / 0..nbx-1), the
            // single-cover ones after them
            uint32_t nbe = 0, nbx = 0;
            for (Member &m : s.members)
                if (!m.single)
                    m.index = m.embed ? nbe++ : nbx++;
            {
                uint32_t ie = nbe, ix = nbx;
                for (Member &m : s.members)
                    if (m.single)
                        m.index = m.embed ? ie++ : ix++;
            }
            for (const Member &m : s.members) {
                if (m.single)
                    continue;
                stego_desc d;
                std::memset(&d, 0, sizeof(d));
                d.cover = m.p.req.cover;
                d.stego = m.p.req.stego;
                d.msg = m.p.req.msg;
                d.cover_bytes = m.p.req.cover_bytes;
                d.msg_bytes = m.p.req.msg_bytes;
                d.msg_len = m.p.req.msg_len;
                d.flags = m.p.req.flags;
                d.geom = m.p.req.geom;
                (m.embed ? s.h_desc_e : s.h_desc_x)[m.index] = d;
            }
            int st = STEGO_OK;
            if (ne) {
                if (nbe && cudaMemcpyAsync(s.d_desc_e, s.h_desc_e, sizeof(stego_desc) * nbe,
                                           cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
                    st = STEGO_E_CUDA;
                if (st == STEGO_OK && nbe)
                    st = stego_embed_batched(s.d_desc_e, nbe, s.d_res_e, STEGO_FUSE_STATS,
                                             &cfg.tune_embed, s.d_ws_e, s.ws_bytes, s.stream);
                if (st == STEGO_OK && ne > nbe)
                    st = launch_singles(s, true);
                if (st == STEGO_OK &&
                    cudaMemcpyAsync(s.h_res_e, s.d_res_e, sizeof(stego_result) * ne,
                                    cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
                    st = STEGO_E_CUDA;
            }
            if (nx && st == STEGO_OK) {
                if (nbx && cudaMemcpyAsync(s.d_desc_x, s.h_desc_x, sizeof(stego_desc) * nbx,
                                           cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
                    st = STEGO_E_CUDA;
                if (st == STEGO_OK && nbx)
                    st = stego_extract_batched(s.d_desc_x, nbx, s.d_res_x, 0, &cfg.tune_extract,
                                               s.d_ws_x, s.ws_bytes, s.stream);
                if (st == STEGO_OK && nx > nbx)
                    st = launch_singles(s, false);
                if (st == STEGO_OK &&
                    cudaMemcpyAsync(s.h_res_x, s.d_res_x, sizeof(stego_result) * nx,
                                    cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
                    st = STEGO_E_CUDA;
            }
            s.launch_status = st;
            if (cudaEventRecord(s.done, s.stream) != cudaSuccess && s.launch_status == STEGO_OK)
                s.launch_status = STEGO_E_CUDA;
            s.busy = true;
            t_last_launch = now();
            {
                std::lock_guard<std::mutex> lk(mu);
                ++batches;
            }
            any = true;
        }
        return any;
    }

    void loop()
    {
        cudaSetDevice(device);
#ifdef __linux__
        // this thread's sleeps end within 1 us of their time instead of the
        // default 50 us timer slack (a per-thread setting)
        prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
        for (;;) {
            const bool a = reap();
            const bool b = dispatch();
            std::unique_lock<std::mutex> lk(mu);
            bool busy = false;
            for (const Slot &s : slots)
                busy = busy || s.busy;
            if (stop && queue.empty() && !busy)
                break;
            if (!a && !b) {
                if (busy) {
                    // batches in flight: poll their events at once for the
                    // first 50 us after a launch (where most batches end),
                    // then every 2 us without holding a core
                    lk.unlock();
                    if (now() - t_last_launch < 50e-6)
                        std::this_thread::yield();
                    else
                        std::this_thread::sleep_for(std::chrono::microseconds(2));
                } else {
                    cv_work.wait_for(lk, std::chrono::milliseconds(2));
                }
            }
        }
    }
};

extern "C" {

uint64_t stego_server_arena_bytes(const stego_server_config *cfg)
{
    if (!config_ok(cfg))
        return 0;
    return slot_bytes(cfg->max_batch) * cfg->slots;
}

int stego_server_create(const stego_server_config *cfg, void *d_arena, uint64_t arena_bytes,
                        stego_server **out)
{
    if (!out || !config_ok(cfg) || !d_arena || ((uintptr_t)d_arena & 255u))
        return STEGO_E_INVAL;
    *out = nullptr;
    if (arena_bytes < stego_server_arena_bytes(cfg))
        return STEGO_E_NOMEM;
    stego_server *s = new stego_server;
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->t0 = Clock::now();
    s->slots.resize(cfg->slots);
    const uint32_t mb = cfg->max_batch;
    const uint64_t dsz = round256(sizeof(stego_desc) * (uint64_t)mb);
    const uint64_t rsz = round256(sizeof(stego_result) * (uint64_t)mb);
    const uint64_t wsz = round256(stego_batched_workspace_bytes(mb));
    char *base = (char *)d_arena;
    int st = STEGO_OK;
    for (uint32_t i = 0; i < cfg->slots && st == STEGO_OK; ++i) {
        Slot &sl = s->slots[i];
        char *p = base + (uint64_t)i * slot_bytes(mb);
        sl.d_desc_e = (stego_desc *)p;
        p += dsz;
        sl.d_desc_x = (stego_desc *)p;
        p += dsz;
        sl.d_res_e = (stego_result *)p;
        p += rsz;
        sl.d_res_x = (stego_result *)p;
        p += rsz;
        sl.d_ws_e = p;
        p += wsz;
        sl.d_ws_x = p;
        sl.ws_bytes = wsz;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_desc_e, dsz, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_desc_x, dsz, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_res_e, rsz, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_res_x, rsz, cudaHostAllocDefault) != cudaSuccess)
            st = STEGO_E_CUDA;
        sl.members.reserve(mb);
    }
    if (st != STEGO_OK) {
        cudaGetLastError();
        stego_server_destroy(s);
        return st;
    }
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return STEGO_OK;
}

double stego_server_clock(stego_server *s) { return s ? s->now() : 0.0; }

int stego_server_submit(stego_server *s, const stego_request *reqs, uint32_t n)
{
    if (!s || (n && !reqs))
        return STEGO_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop)
            return STEGO_E_INVAL;
        const double t = s->now();
        for (uint32_t i = 0; i < n; ++i) {
            Pending p;
            p.req = reqs[i];
            p.t_submit = t;
            p.bytes = request_bytes(reqs[i]);
            s->queue.push_back(p);
            ++s->outstanding;
        }
    }
    s->cv_work.notify_one();
    return STEGO_OK;
}

int stego_server_poll(stego_server *s, stego_completion *out, uint32_t max, uint32_t *n_out)
{
    if (!s || !n_out || (max && !out))
        return STEGO_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const uint32_t k = (uint32_t)std::min<size_t>(max, s->done.size());
    for (uint32_t i = 0; i < k; ++i)
        out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *n_out = k;
    return STEGO_OK;
}

int stego_server_drain(stego_server *s, double timeout_s)
{
    if (!s)
        return STEGO_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s));
    while (s->outstanding > 0)
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && s->outstanding > 0)
            return STEGO_E_TIMEOUT;
    return STEGO_OK;
}

int stego_server_stats(stego_server *s, uint64_t *batches, uint64_t *outstanding,
                       uint64_t *peak_in_flight_bytes)
{
    if (!s)
        return STEGO_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (batches)
        *batches = s->batches;
    if (outstanding)
        *outstanding = s->outstanding;
    if (peak_in_flight_bytes)
        *peak_in_flight_bytes = s->peak_in_flight;
    return STEGO_OK;
}

int stego_server_run_open_loop(stego_server *s, const stego_request *reqs,
                               const double *arrival_s, uint32_t n, stego_completion *out,
                               double timeout_s)
{
    if (!s || (n && (!reqs || !arrival_s || !out)))
        return STEGO_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->outstanding || !s->done.empty())
            return STEGO_E_INVAL; // the runner owns the server while it runs
    }
    const double t0 = s->now();
    for (uint32_t i = 0; i < n; ++i) {
        const double due = t0 + arrival_s[i];
        for (;;) {
            const double gap = due - s->now();
            if (gap <= 0)
                break;
            if (gap > 200e-6)
                std::this_thread::sleep_for(std::chrono::duration<double>(gap - 100e-6));
            else
                std::this_thread::yield();
        }
        Pending p;
        p.req = reqs[i];
        p.req.tag = i;
        p.t_submit = due; // latency counts from the scheduled arrival
        p.bytes = request_bytes(reqs[i]);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->queue.push_back(p);
            ++s->outstanding;
        }
        s->cv_work.notify_one();
    }
    const int st = stego_server_drain(s, timeout_s);
    std::lock_guard<std::mutex> lk(s->mu);
    for (const stego_completion &c : s->done)
        if (c.tag < n)
            out[c.tag] = c;
    s->done.clear();
    return st;
}

int stego_server_destroy(stego_server *s)
{
    if (!s)
        return STEGO_OK;
    if (s->th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->th.join();
    }
    for (Slot &sl : s->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        if (sl.done)
            cudaEventDestroy(sl.done);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_desc_e);
        cudaFreeHost(sl.h_desc_x);
        cudaFreeHost(sl.h_res_e);
        cudaFreeHost(sl.h_res_x);
    }
    delete s;
    return STEGO_OK;
}

} // extern "C"
