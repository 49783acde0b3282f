// Serving: a request loop around the solvers.  Requests (Isaacs grids,
// finite games given as tables, random games given by a seed) are queued in
// arrival order and admitted to worker slots as slots and device memory free
// up; every slot owns a CUDA stream and a solver whose grid-wide launches are
// capped to a share of the GPU, so the work of the requests in flight
// overlaps on the device.  Small games (below the grid-wide threshold) waiting
// together with the same action counts are solved as one batch by a single
// persistent launch (one thread block per game).  Each request's hierarchy and
// policies stay resident on the device for its whole policy iteration; its
// value and policies are copied back to host memory when it completes.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "solver.cuh"

namespace gs {

namespace {

struct Request {
    int64_t id = 0;
    gs_request spec{};
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<double> prob, reward;
    size_t mem = 0;
    int state = 0;                 // 0 queued, 1 running, 2 done
    gs_status status = GS_OK;
    double t_submit = 0, t_start = 0, t_end = 0;
    gs_solve_stats stats{};
    std::vector<double> v;
    std::vector<uint8_t> alpha, beta;
    int64_t n = 0;
    int m1 = 0;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Successors per row of a random-game request (0 = 8).
int succ_of(const gs_request& r) { return r.k > 0 ? r.k : 8; }

// Device bytes a request is expected to hold while it runs, without its
// table (added by the caller for tables given in memory).  A random game
// holds its drawn table twice while it is set.
size_t estimate_bytes(const gs_request& r) {
    if (r.kind == 1) {
        const size_t n = (size_t)r.side * r.side;
        return n * 220 + (64 << 10);
    }
    const size_t rows = (size_t)r.n * r.m1 * r.m2;
    // per row: leakage, reward, policy copies; per state: vectors and the
    // grid kernel's slot-major copy of the selected rows (8 entries)
    const size_t base = rows * 32 + (size_t)r.n * 200 + (64 << 10);
    return r.kind == 3 ? base + 2 * rows * (8 + 12 * (size_t)succ_of(r)) : base;
}

// Games solved together by one batched launch: below the threshold where a
// game alone takes the whole grid, so the batch runs the kernel each of them
// would run alone.
constexpr int kServeBatchMax = 256;
bool batchable(const Request& R) {
    return (R.spec.kind == 2 || R.spec.kind == 3) && R.spec.n < kGameGridMinStates;
}
bool same_batch(const Request& a, const Request& b) {
    return a.spec.kind == b.spec.kind && a.spec.m1 == b.spec.m1 && a.spec.m2 == b.spec.m2 &&
           (a.spec.kind == 2 || succ_of(a.spec) == succ_of(b.spec));
}

}  // namespace

}  // namespace gs

struct gs_server {
    gs_options opt;
    int slots = 1;
    size_t budget = 0;
    size_t in_use = 0;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::deque<std::shared_ptr<gs::Request>> pending;
    std::unordered_map<int64_t, std::shared_ptr<gs::Request>> all;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_id = 1;
    int running = 0;
};

namespace gs {

namespace {

void run_request(gs_solver* solver, Request& R) {
    const gs_request& q = R.spec;
    gs_status st;
    if (q.kind == 1) {
        st = gamesolve_set_isaacs_grid(solver, q.side, q.variant, q.seed, nullptr);
        R.n = (int64_t)q.side * q.side;
        R.m1 = q.variant == 1 ? 5 : 4;
    } else if (q.kind == 3) {
        st = gamesolve_set_random_game(solver, q.n, q.m1, q.m2, succ_of(q), q.seed, q.mu);
        R.n = q.n;
        R.m1 = q.m1;
    } else if (q.flags & GS_REQ_BORROW) {
        st = gamesolve_set_game(solver, q.n, q.m1, q.m2, q.row_ptr, q.col, q.prob, q.reward, q.mu);
        R.n = q.n;
        R.m1 = q.m1;
    } else {
        st = gamesolve_set_game(solver, q.n, q.m1, q.m2, R.row_ptr.data(), R.col.data(),
                                R.prob.data(), R.reward.data(), q.mu);
        R.n = q.n;
        R.m1 = q.m1;
    }
    if (st == GS_OK) {
        st = gamesolve_solve(solver, &R.stats);
        if (st == GS_OK || st == GS_ENOTCONV) {
            R.v.resize(R.n);
            R.alpha.resize(R.n);
            R.beta.resize((size_t)R.n * R.m1);
            gs_status g1 = gamesolve_get_value(solver, R.v.data(), R.n);
            gs_status g2 = gamesolve_get_policy(solver, R.alpha.data(), R.beta.data());
            if (g1 != GS_OK) st = g1;
            else if (g2 != GS_OK) st = g2;
        }
    }
    R.status = st;
}

// Several small games of equal kind and action counts as one batch
// (gamesolve_set_game_batch); results, statistics and status per request.
// A batch the library rejects (a bad table among them) is run request by
// request, so that each gets its own status.
void run_batch(gs_solver* solver, cudaStream_t stream, std::vector<std::shared_ptr<Request>>& B) {
    const int count = (int)B.size();
    const gs_request& q0 = B[0]->spec;
    const int m1 = q0.m1, m2 = q0.m2;
    std::vector<int64_t> off(count + 1, 0);
    std::vector<double> mu(count);
    for (int g = 0; g < count; ++g) {
        off[g + 1] = off[g] + B[g]->spec.n;
        mu[g] = B[g]->spec.mu;
    }
    const int64_t rows = off[count] * m1 * m2;
    gs_status st = GS_OK;
    if (q0.kind == 3) {
        // drawn on the device into one concatenated table
        const int k = succ_of(q0);
        int64_t* rp = nullptr;
        int32_t* col = nullptr;
        double *prob = nullptr, *rew = nullptr;
        bool ok = cudaMalloc(&rp, sizeof(int64_t) * (rows + 1)) == cudaSuccess &&
                  cudaMalloc(&col, sizeof(int32_t) * rows * k) == cudaSuccess &&
                  cudaMalloc(&prob, sizeof(double) * rows * k) == cudaSuccess &&
                  cudaMalloc(&rew, sizeof(double) * rows) == cudaSuccess;
        if (ok) {
            try {
                for (int g = 0; g < count; ++g) {
                    const int64_t r0 = off[g] * m1 * m2;
                    launch_random_game(B[g]->spec.n, m1, m2, k, B[g]->spec.seed, rp + r0, col + r0 * k,
                                       prob + r0 * k, rew + r0, stream, r0 * k);
                }
            } catch (const Error&) {
                ok = false;
            }
        }
        ok = ok && cudaStreamSynchronize(stream) == cudaSuccess;
        st = ok ? gamesolve_set_game_batch(solver, count, m1, m2, off.data(), rp, col, prob, rew, mu.data())
                : GS_ECUDA;
        cudaStreamSynchronize(stream);
        cudaFree(rp);
        cudaFree(col);
        cudaFree(prob);
        cudaFree(rew);
        cudaGetLastError();
    } else {
        // tables in memory: concatenated on the host (columns stay per game)
        std::vector<int64_t> rp(rows + 1, 0);
        std::vector<int32_t> col;
        std::vector<double> prob, rew(rows);
        int64_t r0 = 0;
        bool bad = false;
        for (int g = 0; g < count && !bad; ++g) {
            Request& R = *B[g];
            const gs_request& q = R.spec;
            const int64_t rg = q.n * m1 * m2;
            std::vector<int64_t> rpg;
            const int64_t* rpp = R.row_ptr.data();
            const int32_t* cp = R.col.data();
            const double *pp = R.prob.data(), *wp = R.reward.data();
            std::vector<int32_t> cg;
            std::vector<double> pg, wg;
            if (q.flags & GS_REQ_BORROW) {   // borrowed: host or device memory
                rpg.resize(rg + 1);
                cudaMemcpy(rpg.data(), q.row_ptr, sizeof(int64_t) * (rg + 1), cudaMemcpyDefault);
                const int64_t nz = rpg[rg];
                if (rpg[0] != 0 || nz < 0 || nz > ((int64_t)1 << 40)) {
                    bad = true;
                    break;
                }
                cg.resize(nz);
                pg.resize(nz);
                wg.resize(rg);
                cudaMemcpy(cg.data(), q.col, sizeof(int32_t) * nz, cudaMemcpyDefault);
                cudaMemcpy(pg.data(), q.prob, sizeof(double) * nz, cudaMemcpyDefault);
                cudaMemcpy(wg.data(), q.reward, sizeof(double) * rg, cudaMemcpyDefault);
                rpp = rpg.data();
                cp = cg.data();
                pp = pg.data();
                wp = wg.data();
            }
            if (rpp[0] != 0 || rpp[rg] < 0 ||
                (!(q.flags & GS_REQ_BORROW) && rpp[rg] != (int64_t)R.col.size())) {
                bad = true;   // the library reports it when the request runs alone
                break;
            }
            const int64_t base = (int64_t)col.size(), nz = rpp[rg];
            for (int64_t r = 0; r < rg; ++r) rp[r0 + r + 1] = base + rpp[r + 1];
            col.insert(col.end(), cp, cp + nz);
            prob.insert(prob.end(), pp, pp + nz);
            std::copy(wp, wp + rg, rew.begin() + r0);
            r0 += rg;
        }
        if (bad) st = GS_EINVAL;
        else if (cudaGetLastError() != cudaSuccess) st = GS_ECUDA;
        else st = gamesolve_set_game_batch(solver, count, m1, m2, off.data(), rp.data(),
                                           col.empty() ? (const int32_t*)rp.data() : col.data(),
                                           prob.empty() ? (const double*)rew.data() : prob.data(),
                                           rew.data(), mu.data());
    }
    if (st == GS_EINVAL) {
        for (auto& R : B) run_request(solver, *R);
        return;
    }
    gs_solve_stats total{};
    if (st == GS_OK) st = gamesolve_solve(solver, &total);
    if (st == GS_OK || st == GS_ENOTCONV) {
        std::vector<double> v(off[count]);
        std::vector<uint8_t> alpha(off[count]), beta((size_t)off[count] * m1);
        std::vector<int32_t> gst(4 * (size_t)count);
        std::vector<double> res(count);
        gs_status g1 = gamesolve_get_value(solver, v.data(), off[count]);
        if (g1 == GS_OK) g1 = gamesolve_get_policy(solver, alpha.data(), beta.data());
        if (g1 == GS_OK) g1 = gamesolve_get_batch_stats(solver, gst.data(), res.data());
        for (int g = 0; g < count; ++g) {
            Request& R = *B[g];
            R.n = R.spec.n;
            R.m1 = m1;
            if (g1 != GS_OK) {
                R.status = g1;
                continue;
            }
            R.v.assign(v.begin() + off[g], v.begin() + off[g + 1]);
            R.alpha.assign(alpha.begin() + off[g], alpha.begin() + off[g + 1]);
            R.beta.assign(beta.begin() + off[g] * m1, beta.begin() + off[g + 1] * m1);
            R.stats = total;
            R.stats.outer = gst[4 * g];
            R.stats.systems = gst[4 * g + 1];
            R.stats.cycles = gst[4 * g + 2];
            R.stats.converged = gst[4 * g + 3];
            R.stats.res_inf = res[g];
            R.status = R.stats.converged ? GS_OK : GS_ENOTCONV;
        }
        return;
    }
    for (auto& R : B) R->status = st;
}

void worker(gs_server* S, int slot) {
    cudaSetDevice(S->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    gs_options o = S->opt;
    o.stream = stream;
    if (o.grid_blocks == 0) {
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
        o.grid_blocks = std::max(1, 2 * sms / S->slots);
    }
    gs_solver* solver = nullptr;
    const gs_status created = gamesolve_create(&solver, &o);
    while (true) {
        std::vector<std::shared_ptr<Request>> B;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->work_cv.wait(lk, [&] {
                if (S->stop) return true;
                if (S->pending.empty()) return false;
                const size_t need = S->pending.front()->mem;
                return S->in_use + need <= S->budget || S->running == 0;
            });
            if (S->stop) break;
            B.push_back(S->pending.front());
            S->pending.pop_front();
            S->in_use += B[0]->mem;
            // small games waiting with the same kind and action counts join it
            if (batchable(*B[0])) {
                for (auto it = S->pending.begin(); it != S->pending.end() && (int)B.size() < kServeBatchMax;) {
                    if (batchable(**it) && same_batch(*B[0], **it) && S->in_use + (*it)->mem <= S->budget) {
                        S->in_use += (*it)->mem;
                        B.push_back(*it);
                        it = S->pending.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            ++S->running;
            const double t = now_s(S->t0);
            for (auto& R : B) {
                R->state = 1;
                R->t_start = t;
            }
        }
        if (created != GS_OK) {
            for (auto& R : B) R->status = created;
        } else if (B.size() == 1) {
            run_request(solver, *B[0]);
        } else {
            run_batch(solver, stream, B);
        }
        for (auto& R : B) {
            R->row_ptr.clear();
            R->row_ptr.shrink_to_fit();
            R->col.clear();
            R->col.shrink_to_fit();
            R->prob.clear();
            R->prob.shrink_to_fit();
            R->reward.clear();
            R->reward.shrink_to_fit();
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double t = now_s(S->t0);
            for (auto& R : B) {
                R->t_end = t;
                R->state = 2;
                S->in_use -= R->mem;
            }
            --S->running;
        }
        S->work_cv.notify_all();
        S->done_cv.notify_all();
    }
    if (solver) gamesolve_destroy(solver);
    if (stream) cudaStreamDestroy(stream);
    (void)slot;
}

void fill_info(const Request& R, gs_ticket_info* info) {
    if (!info) return;
    std::memset(info, 0, sizeof *info);
    info->state = R.state;
    info->status = R.status;
    info->t_submit = R.t_submit;
    info->t_start = R.t_start;
    info->t_end = R.t_end;
    info->n = R.n;
    info->stats = R.stats;
}

}  // namespace

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gamesolve_server_create(gs_server** out, const gs_options* opt, int32_t slots,
                                  uint64_t mem_budget) {
    if (!out || slots < 1 || slots > 64) {
        set_last_error("server_create: invalid argument");
        return GS_EINVAL;
    }
    gs_options o;
    if (opt) o = *opt;
    else gamesolve_default_options(&o);
    gs_solver* probe = nullptr;
    const gs_status st = gamesolve_create(&probe, &o);   // validates the options and the device
    if (st != GS_OK) return st;
    gamesolve_destroy(probe);
    auto* S = new gs_server();
    S->opt = o;
    S->slots = slots;
    cudaGetDevice(&S->device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    S->budget = mem_budget ? (size_t)mem_budget : free_b / 2;
    S->t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < slots; ++k) S->workers.emplace_back(worker, S, k);
    *out = S;
    return GS_OK;
}

gs_status gamesolve_server_submit(gs_server* S, const gs_request* req, int64_t* ticket) {
    if (!S || !req || !ticket) return GS_EINVAL;
    auto R = std::make_shared<Request>();
    R->spec = *req;
    if (req->kind == 1) {
        if (req->side < 1 || ((req->side + 1) & req->side) != 0 || (req->variant != 0 && req->variant != 1)) {
            set_last_error("server_submit: side must be 2^k - 1 and variant 0 or 1");
            return GS_EINVAL;
        }
    } else if (req->kind == 2) {
        if (req->n < 1 || req->m1 < 1 || req->m1 > kGameMaxM1 || req->m2 < 1 || req->m2 > kGameMaxM2 ||
            !req->row_ptr || !req->col || !req->prob || !req->reward) {
            set_last_error("server_submit: invalid game");
            return GS_EINVAL;
        }
        const int64_t rows = req->n * req->m1 * req->m2;
        int64_t nnz = 0;
        if (cudaMemcpy(&nnz, req->row_ptr + rows, sizeof nnz, cudaMemcpyDefault) != cudaSuccess ||
            nnz < 0) {
            cudaGetLastError();
            set_last_error("server_submit: unreadable row_ptr");
            return GS_EINVAL;
        }
        if (req->flags & GS_REQ_BORROW) {
            R->mem = estimate_bytes(*req) + (size_t)nnz * 24;
            goto queued;
        }
        // the request owns a host copy of its table until it has run
        R->row_ptr.resize(rows + 1);
        R->col.resize(nnz);
        R->prob.resize(nnz);
        R->reward.resize(rows);
        cudaMemcpy(R->row_ptr.data(), req->row_ptr, sizeof(int64_t) * (rows + 1), cudaMemcpyDefault);
        cudaMemcpy(R->col.data(), req->col, sizeof(int32_t) * nnz, cudaMemcpyDefault);
        cudaMemcpy(R->prob.data(), req->prob, sizeof(double) * nnz, cudaMemcpyDefault);
        cudaMemcpy(R->reward.data(), req->reward, sizeof(double) * rows, cudaMemcpyDefault);
        if (cudaGetLastError() != cudaSuccess) {
            set_last_error("server_submit: copying the table failed");
            return GS_EINVAL;
        }
        R->spec.row_ptr = nullptr;
        R->spec.col = nullptr;
        R->spec.prob = nullptr;
        R->spec.reward = nullptr;
    } else if (req->kind == 3) {
        if (!random_game_args_ok(req->n, req->m1, req->m2, succ_of(*req)) || req->k < 0 ||
            !(req->mu > 0.0 && req->mu < 1.0)) {
            set_last_error("server_submit: invalid random game");
            return GS_EINVAL;
        }
    } else {
        set_last_error("server_submit: kind must be 1 (Isaacs), 2 (game) or 3 (random game)");
        return GS_EINVAL;
    }
    R->mem = estimate_bytes(*req) + (req->kind == 2 ? R->col.size() * 24 : 0);
queued:
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R->id = S->next_id++;
        R->t_submit = now_s(S->t0);
        S->pending.push_back(R);
        S->all[R->id] = R;
        *ticket = R->id;
    }
    S->work_cv.notify_all();
    return GS_OK;
}

gs_status gamesolve_server_poll(gs_server* S, int64_t ticket, gs_ticket_info* info) {
    if (!S) return GS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return GS_EINVAL;
    fill_info(*it->second, info);
    return GS_OK;
}

gs_status gamesolve_server_wait(gs_server* S, int64_t ticket, gs_ticket_info* info) {
    if (!S) return GS_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return GS_EINVAL;
    std::shared_ptr<Request> R = it->second;
    S->done_cv.wait(lk, [&] { return R->state == 2; });
    fill_info(*R, info);
    return GS_OK;
}

gs_status gamesolve_server_result(gs_server* S, int64_t ticket, double* v_out, int64_t n,
                                  uint8_t* alpha, uint8_t* beta) {
    if (!S) return GS_EINVAL;
    std::shared_ptr<Request> R;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) return GS_EINVAL;
        R = it->second;
        if (R->state != 2) return GS_ESTATE;
        S->all.erase(it);
    }
    if (R->status != GS_OK && R->status != GS_ENOTCONV) return R->status;
    if (n != R->n) {
        set_last_error("server_result: n = %lld, request has %lld states", (long long)n,
                       (long long)R->n);
        return GS_EINVAL;
    }
    if (v_out) cudaMemcpy(v_out, R->v.data(), sizeof(double) * n, cudaMemcpyDefault);
    if (alpha) cudaMemcpy(alpha, R->alpha.data(), n, cudaMemcpyDefault);
    if (beta) cudaMemcpy(beta, R->beta.data(), (size_t)n * R->m1, cudaMemcpyDefault);
    return R->status;
}

void gamesolve_server_destroy(gs_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->work_cv.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
}

}  // extern "C"
