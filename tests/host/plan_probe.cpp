// Host-logic probe for the CPU tests: prints the planner's integer description
// of one discretisation (node positions, the node bands, the node ranges N^(i)
// and the exactness ranges J^(i) of Sect. 4.1 and, for a closed curve, the
// collocation nodes).  Links only the planner; no GPU
// is touched.  Usage: plan_probe n_elems degree n_ref closed
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../paper_1703_10016_gb300/csrc/igs_internal.h"

static void row(const char* name, const std::vector<int>& v) {
    std::printf("%s", name);
    for (int x : v) std::printf(" %d", x);
    std::printf("\n");
}

int main(int argc, char** argv) {
    if (argc != 5) return 1;
    const int n = std::atoi(argv[1]), d = std::atoi(argv[2]), nref = std::atoi(argv[3]), closed = std::atoi(argv[4]);
    igs::Plan P;
    std::string err;
    if (igs::build_plan(P, 0.0, 1.0, n, d, nref, closed, err) != IGS_OK) {
        std::printf("error %s\n", err.c_str());
        return 2;
    }
    std::printf("den %d\n", P.den);
    row("pos", P.pos_num);
    row("lo", P.lo);
    row("hi", P.hi);
    row("jfirst", P.jfirst);
    row("member", P.member);
    row("jlo1", P.jlo1);
    row("jhi1", P.jhi1);
    row("jlo2", P.jlo2);
    row("jhi2", P.jhi2);
    if (closed) {
        std::vector<int> c;
        if (igs::collocation_nodes(P, c, err) == IGS_OK) row("colloc", c);
        else std::printf("colloc_error %s\n", err.c_str());
    }
    return 0;
}
