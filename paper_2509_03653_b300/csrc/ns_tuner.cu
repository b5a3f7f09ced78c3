// ns_tuner.cu -- the autotuners' cache file.
//
// One JSON object of entries, one entry per line:
//   "<gpu name>|<kind>|<shape>": {<field>: <number or string>, ...}
// Kinds so far: "batch" (ns_batch_tune's launch parameters) and "path"
// (ns_path_tune's choice between the sort and hash paths).  Entries of a
// kind a reader does not know are kept verbatim when the file is rewritten,
// so the tuners never erase one another's results.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "ns_api_internal.h"

namespace ns {

std::string gpu_name(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    std::string n(prop.name, strnlen(prop.name, sizeof prop.name));
    for (char& ch : n)
        if (ch == '"' || ch == '|' || ch == '\\' || ch == '\n') ch = '_';
    return n;
}

std::map<std::string, std::string> tuner_load(const std::string& path) {
    std::map<std::string, std::string> m;
    if (path.empty()) return m;
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return m;
    char line[2048];
    while (fgets(line, sizeof line, f)) {
        char* q1 = strchr(line, '"');
        if (!q1) continue;
        char* q2 = strchr(q1 + 1, '"');
        if (!q2) continue;
        char* b0 = strchr(q2, '{');
        char* b1 = b0 ? strchr(b0, '}') : nullptr;
        if (!b0 || !b1) continue;
        m[std::string(q1 + 1, q2)] = std::string(b0, b1 + 1);
    }
    fclose(f);
    return m;
}

void tuner_store(const std::string& path, const std::map<std::string, std::string>& m) {
    if (path.empty()) return;
    const std::string tmp = path + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto& kv : m) fprintf(f, "  \"%s\": %s%s\n", kv.first.c_str(), kv.second.c_str(), ++i < m.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path.c_str());
}

bool json_number(const std::string& obj, const char* name, double* v) {
    const std::string pat = std::string("\"") + name + "\":";
    const size_t p = obj.find(pat);
    if (p == std::string::npos) return false;
    const char* s = obj.c_str() + p + pat.size();
    char* e = nullptr;
    const double x = strtod(s, &e);
    if (e == s) return false;
    *v = x;
    return true;
}

bool json_string(const std::string& obj, const char* name, std::string* v) {
    const std::string pat = std::string("\"") + name + "\":";
    size_t p = obj.find(pat);
    if (p == std::string::npos) return false;
    p = obj.find('"', p + pat.size());
    if (p == std::string::npos) return false;
    const size_t q = obj.find('"', p + 1);
    if (q == std::string::npos) return false;
    *v = obj.substr(p + 1, q - p - 1);
    return true;
}

}  // namespace ns
