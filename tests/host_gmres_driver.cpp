// Test driver for csrc/host_gmres.h: reads n, max_iter, tol, fail_after, the
// n x n column-major matrix A and the right side b from a binary file; solves
// A x = b with host_gmres (the operator fails after fail_after applications
// when fail_after >= 0) and writes status, iterations, relative residual and
// x to the output file.
#include <cstdio>
#include <vector>

#include "../paper_2004_08669_gb300/csrc/host_gmres.h"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = std::fopen(argv[1], "rb");
    if (!in) return 3;
    int hdr[3];
    double tol;
    if (std::fread(hdr, sizeof(int), 3, in) != 3 || std::fread(&tol, sizeof(double), 1, in) != 1) return 4;
    const int n = hdr[0], max_iter = hdr[1], fail_after = hdr[2];
    std::vector<double> A((size_t)n * n), b(n), x;
    if (std::fread(A.data(), sizeof(double), A.size(), in) != A.size()) return 5;
    if (std::fread(b.data(), sizeof(double), b.size(), in) != b.size()) return 6;
    std::fclose(in);
    int applied = 0;
    auto op = [&](const std::vector<double>& v, std::vector<double>& w) -> bool {
        if (fail_after >= 0 && applied >= fail_after) return false;
        ++applied;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += A[i + (size_t)n * j] * v[j];
            w[i] = s;
        }
        return true;
    };
    int iters = 0;
    double res = 0.0;
    const int st = ctm::host_gmres(op, b, x, tol, max_iter, &iters, &res);
    FILE* out = std::fopen(argv[2], "wb");
    if (!out) return 7;
    const int o[2] = {st, iters};
    std::fwrite(o, sizeof(int), 2, out);
    std::fwrite(&res, sizeof(double), 1, out);
    std::fwrite(x.data(), sizeof(double), x.size(), out);
    std::fclose(out);
    return 0;
}
