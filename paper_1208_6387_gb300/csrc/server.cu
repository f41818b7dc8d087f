// Serving: continuous batching of whole structures over a resident pattern library (include/fetirp.h).
// Written on the public C ABI: every slot is a worker thread driving a child context of the library.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fetirp.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  // structure (owned copies)
  int32_t n_occ = 0;
  std::vector<int32_t> pattern_id, link_offset, local_node, lambda_row, group_of_occ;
  std::vector<int8_t> global_comp, sign;
  std::vector<double> rot, f_global, c;
  std::vector<int64_t> f_offset;
  int64_t n_lambda = 0;
  int32_t k = 0;
  int64_t mem = 0;   // device-memory estimate
  // result
  bool done = false;
  fetirp_status status = FETIRP_OK;
  std::vector<double> lambda, u;
  fetirp_stats stats{};
  Clock::time_point t_submit, t_done;
};

// Device memory a structure will hold while it is solved: work blocks, direction history (capped by the slot
// options), local traces and products, per-pattern loads and solutions.
int64_t estimate_bytes(const Request& r, const fetirp_options& o) {
  const double nl = (double)r.n_lambda;
  const int k = r.k > 0 ? r.k : std::max(1, std::min(o.block_k, r.n_occ));
  const double ndofs = (double)r.f_offset.back();
  const double hist = o.history_bytes > 0 ? (double)o.history_bytes
                                          : 2.0 * 8.0 * nl * std::min<double>(nl, (double)o.max_iter * k);
  const double work = 8.0 * nl * (12.0 + 6.0 * k) + 2.0 * 8.0 * ndofs + 5.0 * 8.0 * ndofs / 4.0 * k;
  return (int64_t)(hist + work);
}

}  // namespace

struct fetirp_server_s {
  fetirp_ctx lib = nullptr;
  fetirp_options opt{};
  int64_t budget = 0;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<int64_t, std::unique_ptr<Request>> all;
  int64_t next_ticket = 1;
  int64_t in_use = 0;
  int active = 0;
  bool stop = false;
  int max_batch = 1;   // structures one slot may take together (fetirp_server_set_batching)

  static int32_t width_of(const Request* r, const fetirp_options& o) {
    const int32_t k = r->k > 0 ? r->k : o.block_k;
    return std::max(1, std::min(k, r->n_occ));
  }
  static int32_t single_pattern(const Request* r) {   // the one library pattern of r, or -1
    for (int32_t o = 1; o < r->n_occ; ++o)
      if (r->pattern_id[o] != r->pattern_id[0]) return -1;
    return r->pattern_id[0];
  }

  void worker_loop() {
    fetirp_ctx child = nullptr;
    for (;;) {
      std::vector<Request*> batch;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv_work.wait(lock, [&] {
          if (stop && pending.empty()) return true;
          if (pending.empty()) return false;
          const Request* f = pending.front();
          return active == 0 || in_use + f->mem <= budget;
        });
        if (pending.empty()) break;   // stop requested and queue drained
        Request* r = pending.front();
        pending.pop_front();
        in_use += r->mem;
        batch.push_back(r);
        // continuous batching: queued structures of the same library pattern join this slot's solve while the
        // union stays within 64 multivector columns and the memory budget (they are solved as independent
        // blocks of one structure, so every local-product launch serves all of them)
        const int32_t pat = single_pattern(r);
        int32_t width = width_of(r, opt);
        for (auto it = pending.begin(); max_batch > 1 && pat >= 0 && it != pending.end() &&
                                        (int)batch.size() < max_batch;) {
          Request* q = *it;
          const int32_t wq = width_of(q, opt);
          if (single_pattern(q) == pat && width + wq <= 64 && in_use + q->mem <= budget) {
            batch.push_back(q);
            width += wq;
            in_use += q->mem;
            it = pending.erase(it);
          } else {
            ++it;
          }
        }
        ++active;
      }
      fetirp_status st = FETIRP_OK;
      if (!child) st = fetirp_create_child(lib, &opt, &child);
      if (st == FETIRP_OK) st = fetirp_clear_occurrences(child);
      int64_t row0 = 0;
      std::vector<int64_t> row_off{0}, u_off{0};
      std::vector<int32_t> groups;
      int32_t g0 = 0;
      for (Request* r : batch) {
        for (int32_t o = 0; st == FETIRP_OK && o < r->n_occ; ++o) {
          const int32_t l0 = r->link_offset[o], l1 = r->link_offset[o + 1];
          std::vector<int32_t> rows(r->lambda_row.begin() + l0, r->lambda_row.begin() + l1);
          for (auto& x : rows) x += (int32_t)row0;   // the request's multiplier rows, after the earlier ones
          int32_t id = 0;
          st = fetirp_add_occurrence(child, r->pattern_id[o], r->rot.empty() ? nullptr : &r->rot[9 * (size_t)o],
                                     l1 - l0, r->local_node.data() + l0, r->global_comp.data() + l0, rows.data(),
                                     r->sign.data() + l0, r->f_global.data() + r->f_offset[o], &id);
        }
        const int32_t k = width_of(r, opt);
        for (int32_t o = 0; o < r->n_occ; ++o)
          groups.push_back(g0 + (r->group_of_occ.empty() ? (int32_t)((int64_t)o * k / r->n_occ)
                                                         : std::min(r->group_of_occ[o], k - 1)));
        g0 += k;
        row0 += r->n_lambda;
        row_off.push_back(row0);
        u_off.push_back(u_off.back() + r->f_offset.back());
      }
      const bool explicit_groups = batch.size() > 1 || batch[0]->k > 0 || !batch[0]->group_of_occ.empty();
      if (st == FETIRP_OK && explicit_groups) st = fetirp_set_groups(child, g0, groups.data());
      if (st == FETIRP_OK && batch.size() > 1)
        st = fetirp_set_row_blocks(child, (int32_t)batch.size(), row_off.data());
      std::vector<double> lam, u, c;
      fetirp_stats stats{};
      if (st == FETIRP_OK) {
        lam.resize((size_t)row0);
        u.resize((size_t)u_off.back());
        bool any_c = false;
        for (Request* r : batch) any_c = any_c || !r->c.empty();
        if (any_c) {
          c.assign((size_t)row0, 0.0);
          for (size_t b = 0; b < batch.size(); ++b)
            if (!batch[b]->c.empty()) std::copy(batch[b]->c.begin(), batch[b]->c.end(), c.begin() + row_off[b]);
        }
        st = fetirp_solve(child, row0, c.empty() ? nullptr : c.data(), lam.data(), u.data(), &stats);
      }
      {
        std::lock_guard<std::mutex> lock(mu);
        for (size_t b = 0; b < batch.size(); ++b) {
          Request* r = batch[b];
          r->status = st;
          if (!lam.empty()) {
            r->lambda.assign(lam.begin() + row_off[b], lam.begin() + row_off[b + 1]);
            r->u.assign(u.begin() + u_off[b], u.begin() + u_off[b + 1]);
          }
          r->stats = stats;
          r->done = true;
          r->t_done = Clock::now();
          in_use -= r->mem;
        }
        --active;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (child) fetirp_destroy(child);
  }
};

extern "C" {

fetirp_status fetirp_server_create(fetirp_ctx library, const fetirp_options* slot_opt, int32_t max_slots,
                                   int64_t mem_budget_bytes, fetirp_server* out) {
  if (!library || !out || max_slots < 1 || max_slots > 256 || mem_budget_bytes <= 0) return FETIRP_EINVAL;
  auto srv = std::make_unique<fetirp_server_s>();
  srv->lib = library;
  if (slot_opt) srv->opt = *slot_opt;
  else fetirp_default_options(&srv->opt);
  srv->opt.cuda_stream = nullptr;   // every slot owns its stream
  srv->budget = mem_budget_bytes;
  fetirp_server_s* p = srv.get();
  for (int32_t i = 0; i < max_slots; ++i) p->workers.emplace_back([p] { p->worker_loop(); });
  *out = srv.release();
  return FETIRP_OK;
}

fetirp_status fetirp_server_set_batching(fetirp_server srv, int32_t max_structures) {
  if (!srv || max_structures < 1 || max_structures > 64) return FETIRP_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  srv->max_batch = max_structures;
  return FETIRP_OK;
}

fetirp_status fetirp_server_submit(fetirp_server srv, const fetirp_structure* s, int64_t* ticket) {
  if (!srv || !s || !ticket || s->n_occ < 1 || s->n_lambda < 1 || !s->pattern_id || !s->link_offset ||
      !s->f_offset || !s->f_global)
    return FETIRP_EINVAL;
  auto r = std::make_unique<Request>();
  const int32_t n = s->n_occ;
  const int32_t nl = s->link_offset[n];
  const int64_t nf = s->f_offset[n];
  if (nl < 0 || nf <= 0 || (nl > 0 && (!s->local_node || !s->global_comp || !s->lambda_row || !s->sign)))
    return FETIRP_EINVAL;
  r->n_occ = n;
  r->pattern_id.assign(s->pattern_id, s->pattern_id + n);
  if (s->rot) r->rot.assign(s->rot, s->rot + 9 * (size_t)n);
  r->link_offset.assign(s->link_offset, s->link_offset + n + 1);
  r->local_node.assign(s->local_node, s->local_node + nl);
  r->global_comp.assign(s->global_comp, s->global_comp + nl);
  r->lambda_row.assign(s->lambda_row, s->lambda_row + nl);
  r->sign.assign(s->sign, s->sign + nl);
  r->f_offset.assign(s->f_offset, s->f_offset + n + 1);
  r->f_global.assign(s->f_global, s->f_global + nf);
  r->n_lambda = s->n_lambda;
  if (s->c) r->c.assign(s->c, s->c + s->n_lambda);
  r->k = s->k;
  if (s->group_of_occ) r->group_of_occ.assign(s->group_of_occ, s->group_of_occ + n);
  r->mem = estimate_bytes(*r, srv->opt);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    r->ticket = srv->next_ticket++;
    *ticket = r->ticket;
    srv->pending.push_back(r.get());
    srv->all.emplace(r->ticket, std::move(r));
  }
  srv->cv_work.notify_one();
  return FETIRP_OK;
}

fetirp_status fetirp_server_wait(fetirp_server srv, int64_t ticket, double timeout_s, int32_t* done,
                                 double* lambda_out, double* u_out, fetirp_stats* stats, double* latency_ms) {
  if (!srv || !done) return FETIRP_EINVAL;
  std::unique_lock<std::mutex> lock(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return FETIRP_EINVAL;
  Request* r = it->second.get();
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) srv->cv_done.wait(lock, ready);
  else if (timeout_s > 0) srv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready);
  *done = r->done ? 1 : 0;
  if (!r->done) return FETIRP_OK;
  if (lambda_out && !r->lambda.empty()) std::memcpy(lambda_out, r->lambda.data(), sizeof(double) * r->lambda.size());
  if (u_out && !r->u.empty()) std::memcpy(u_out, r->u.data(), sizeof(double) * r->u.size());
  if (stats) *stats = r->stats;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const fetirp_status st = r->status;
  srv->all.erase(it);
  return st;
}

fetirp_status fetirp_server_poll(fetirp_server srv, int64_t ticket, int32_t* done, double* lambda_out,
                                 double* u_out, fetirp_stats* stats, double* latency_ms) {
  return fetirp_server_wait(srv, ticket, 0.0, done, lambda_out, u_out, stats, latency_ms);
}

void fetirp_server_destroy(fetirp_server srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  delete srv;
}

}  // extern "C"
