// trace.cuh -- the per-kernel-class event tracer behind CWM_TRACE (common.cuh).
#pragma once

#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace cwm {

struct TraceEntry {
  std::string name;
  long long launches;
  double ms;
  double bytes;
};

struct Tracer {
  bool on = false;
  std::string filter;  // category prefix; empty = every category
  std::vector<TraceEntry> entries;
  struct Pending {
    int idx;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // while a stream capture is recorded, scopes land here: their events are re-recorded by
  // every replay of the graph and read back by collect_graph() after each replay
  bool capturing = false;
  std::vector<Pending> graph_pending;
  ~Tracer();
  // after a replay of a graph has completed: fold that graph's scopes in
  void collect(const std::vector<Pending> &scopes);
  // the graph is destroyed: recycle its events
  void release(std::vector<Pending> &scopes);
  bool wants(const char *cat) const;
  int entry(const char *cat);
  cudaEvent_t event();
  void flush();  // waits for the recorded events and folds them into `entries`
};

}  // namespace cwm
