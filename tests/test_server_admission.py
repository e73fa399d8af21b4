"""The request server's admission policy (csrc/hz_admission.h, used by
hz_server.cpp) compiled on its own with the host C++ compiler: first fit in
arrival order against the HBM budget, pass-over counting, and the
starvation guard that stops admissions behind a request passed over too
often.  No GPU is involved."""

import os
import shutil
import subprocess

import pytest

from conftest import ROOT

SRC = r"""
#include <cstdio>
#include <deque>
#include <vector>
#include "hz_admission.h"

struct R { unsigned long long bytes; int passed_over; int id; };

#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main() {
  using hz::first_fit;
  {  // empty queue
    std::deque<R*> q;
    CHECK(first_fit(q, 0, 100, 64) == nullptr);
  }
  {  // the head fits: admitted, nobody passed over
    R a{40, 0, 0}, b{10, 0, 1};
    std::deque<R*> q{&a, &b};
    CHECK(first_fit(q, 0, 100, 64) == &a);
    CHECK(q.size() == 1 && q.front() == &b && b.passed_over == 0);
  }
  {  // the head does not fit: the first that does is admitted, the head passed over once
    R a{100, 0, 0}, b{60, 0, 1}, c{10, 0, 2};
    std::deque<R*> q{&a, &b, &c};
    CHECK(first_fit(q, 50, 100, 64) == &c);
    CHECK(a.passed_over == 1 && b.passed_over == 1 && q.size() == 2);
    CHECK(first_fit(q, 50, 100, 64) == nullptr);  // nothing else fits
    CHECK(a.passed_over == 1 && b.passed_over == 1);  // a failed scan counts nothing
  }
  {  // an exact fit is admitted
    R a{30, 0, 0};
    std::deque<R*> q{&a};
    CHECK(first_fit(q, 70, 100, 64) == &a);
  }
  {  // starvation guard: once the head was passed over max times, nothing behind it is admitted
    R big{90, 0, 0};
    std::vector<R> small(5, R{5, 0, 1});
    std::deque<R*> q{&big};
    for (auto& s : small) q.push_back(&s);
    int admitted = 0;
    for (int k = 0; k < 10; ++k) {
      R* r = first_fit(q, 20, 100, 3);  // 20 in use: big (90) does not fit
      if (r) ++admitted;
    }
    CHECK(admitted == 3 && big.passed_over == 3 && q.front() == &big);
    CHECK(first_fit(q, 0, 100, 3) == &big);  // it is next once memory frees
    CHECK(first_fit(q, 0, 100, 3) == &small[3]);
  }
  {  // arrival order among requests that fit
    R a{10, 0, 0}, b{10, 0, 1};
    std::deque<R*> q{&a, &b};
    CHECK(first_fit(q, 0, 15, 64) == &a);
    CHECK(first_fit(q, 10, 15, 64) == nullptr);
  }
  std::printf("ok\n");
  return 0;
}
"""


def test_first_fit_admission_with_starvation_guard(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "admission.cpp"
    src.write_text(SRC)
    exe = tmp_path / "admission"
    inc = os.path.join(ROOT, "paper_2606_21695_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
