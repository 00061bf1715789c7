// Host side of the autotuner: the choice among measured configurations and
// their cache file.  No device code and no CUDA call: mg_plan_autotune (api.cu)
// measures the candidates on the GPU and hands them to these functions.
//
// A candidate is a way of evolving a job: the arithmetic of its matrix products
// (native FP64, or BF16 digit products with `slices` digits), the Taylor scheme
// of the exponential (degree 18 in five products allowed, or Paterson-Stockmeyer
// only), and for state outputs the action-based path.  Each carries its
// estimated max-abs error over the job's N intervals and its measured device
// time per interval; the choice is the fastest candidate whose error, times a
// safety factor, stays within the caller's tolerance.
//
// Cache file: plain text, one line per tuning,
//   <key> TAB <selected index> TAB <entry>;<entry>;...
// with every entry "precision slices taylor action error us_per_interval
// taylor_target" (entries of six fields read with taylor_target 0).  A
// lookup takes the last line whose key matches (exactly, or by prefix up to a
// '|' boundary for callers that know only the leading fields of the key).
#include "common.cuh"

#include <sys/file.h>
#include <unistd.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <fcntl.h>
#include <string>
#include <vector>

using namespace mg;

namespace {

bool parse_line(const std::string& line, std::string& key, int& sel, std::vector<mg_tune_entry>& ents) {
  const size_t t1 = line.find('\t');
  if (t1 == std::string::npos) return false;
  const size_t t2 = line.find('\t', t1 + 1);
  if (t2 == std::string::npos) return false;
  key = line.substr(0, t1);
  sel = std::atoi(line.substr(t1 + 1, t2 - t1 - 1).c_str());
  ents.clear();
  size_t pos = t2 + 1;
  while (pos < line.size()) {
    size_t end = line.find(';', pos);
    if (end == std::string::npos) end = line.size();
    const std::string f = line.substr(pos, end - pos);
    mg_tune_entry e{};
    int p, s, t, a;
    double err, us, tu = 0.0;
    const int got = std::sscanf(f.c_str(), "%d %d %d %d %lg %lg %lg", &p, &s, &t, &a, &err, &us, &tu);
    if (got == 6 || got == 7) {
      e.precision = p;
      e.slices = s;
      e.taylor = t;
      e.action = a;
      e.error = err;
      e.us_per_interval = us;
      e.taylor_target = got == 7 ? tu : 0.0;
      ents.push_back(e);
    }
    pos = end + 1;
  }
  return sel >= 0 && sel < (int)ents.size();
}

bool key_matches(const std::string& stored, const char* want) {
  const size_t n = std::strlen(want);
  if (stored.size() < n || stored.compare(0, n, want) != 0) return false;
  return stored.size() == n || stored[n] == '|' || (n > 0 && want[n - 1] == '|');
}

}  // namespace

extern "C" {

int mg_tune_select(int n, const mg_tune_entry* e, double tolerance, double safety, int* index) {
  if (n < 1 || !e || !index || !(tolerance > 0.0) || !(safety >= 1.0)) return MG_EINVAL;
  int best = -1;
  for (int i = 0; i < n; ++i) {
    if (!(e[i].us_per_interval > 0.0) || !std::isfinite(e[i].us_per_interval)) continue;
    if (!(e[i].error >= 0.0) || !(e[i].error * safety <= tolerance)) continue;   // NaN errors never qualify
    if (best < 0 || e[i].us_per_interval < e[best].us_per_interval) best = i;
  }
  if (best < 0) {
    set_last_message("no measured configuration meets the tolerance %g (safety factor %g)", tolerance, safety);
    return MG_EUNSUPPORTED;
  }
  *index = best;
  return MG_OK;
}

int mg_tune_cache_store(const char* path, const char* key, int n, const mg_tune_entry* e, int selected) {
  if (!path || !key || !*key || n < 1 || !e || selected < 0 || selected >= n) return MG_EINVAL;
  if (std::strchr(key, '\t') || std::strchr(key, '\n') || std::strchr(key, ';')) return MG_EINVAL;
  std::string line = std::string(key) + "\t" + std::to_string(selected) + "\t";
  char buf[192];
  for (int i = 0; i < n; ++i) {
    std::snprintf(buf, sizeof(buf), "%s%d %d %d %d %.17g %.17g %.17g", i ? ";" : "", e[i].precision, e[i].slices,
                  e[i].taylor, e[i].action, e[i].error, e[i].us_per_interval, e[i].taylor_target);
    line += buf;
  }
  line += "\n";
  const int fd = ::open(path, O_WRONLY | O_CREAT | O_APPEND, 0644);
  if (fd < 0) {
    set_last_message("cannot open the tuning cache %s for appending", path);
    return MG_EINVAL;
  }
  ::flock(fd, LOCK_EX);
  const ssize_t w = ::write(fd, line.data(), line.size());
  ::flock(fd, LOCK_UN);
  ::close(fd);
  if (w != (ssize_t)line.size()) {
    set_last_message("short write to the tuning cache %s", path);
    return MG_EINVAL;
  }
  return MG_OK;
}

int mg_tune_cache_lookup(const char* path, const char* key, mg_tune_entry* out) {
  if (!path || !key || !out) return MG_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return MG_EAGAIN;
  std::string line, k;
  std::vector<mg_tune_entry> ents;
  bool found = false;
  mg_tune_entry hit{};
  char buf[4096];
  while (std::fgets(buf, sizeof(buf), f)) {
    line += buf;
    if (line.empty() || line.back() != '\n') continue;   // a longer line continues
    line.pop_back();
    int sel = -1;
    if (parse_line(line, k, sel, ents) && key_matches(k, key)) {
      hit = ents[sel];
      found = true;
    }
    line.clear();
  }
  std::fclose(f);
  if (!found) return MG_EAGAIN;
  *out = hit;
  return MG_OK;
}

}  // extern "C"
