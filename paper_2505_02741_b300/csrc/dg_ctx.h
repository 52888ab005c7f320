// dg_ctx.h -- library context: device, configuration, allocator, graphs and
// the serving scheduler.
#pragma once
#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

#include "dg_batch.cuh"

namespace dg {

struct Request {
    uint64_t ticket = 0;
    int32_t gid = 0;
    std::vector<dg_update> ups;
    dg_update_result* res = nullptr;
    uint64_t need_bytes = 0;
    double t_submit = 0.0;
    double t_start = 0.0;  // a worker took it (admitted)
    double t_done = 0.0;
    dg_status status = DG_OK;
    bool done = false;
    std::string error;
};

struct Ctx {
    int device = 0;
    Config cfg;
    DevAlloc alloc;
    cudaStream_t stream = nullptr;
    std::mutex mu;  // graphs map, id counter
    std::map<int32_t, std::unique_ptr<DGraph>> graphs;
    int32_t next_gid = 1;
    std::atomic<uint64_t> launches{0};
    int64_t fin_wait_polls = -1;  // finalize-queue poll limit of the walk (< 0: FIN_SPIN_LIMIT)

    // serving
    std::mutex smu;
    std::condition_variable scv;   // work available / state change
    std::condition_variable dcv;   // request completed
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> tickets;
    std::map<int32_t, bool> busy;  // graph id -> a request of it is running
    uint64_t in_flight_bytes = 0;
    uint64_t next_ticket = 1;
    std::vector<std::thread> workers;
    bool stopping = false;
    int n_workers = 0;

    DGraph& graph(int32_t gid);
};

double now_ms();
void set_last_error(const std::string& msg);  // the text dg_last_error() returns on this thread

}  // namespace dg
