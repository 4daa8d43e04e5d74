// Velocity sets of the engine: D2Q9 (theta = 1/3) and D2Q21 (Table I of the
// paper, theta = 2/3, third row read as (+-2,0),(0,+-2)).  Compile-time tables
// so that every loop over states unrolls and every c_i folds to a constant.
#pragma once

namespace lbm {

template <int Q> struct Lattice;

template <> struct Lattice<9> {
  static constexpr int Q = 9;
  static constexpr int R = 1;  // largest |c| component: streaming / force reach
  static constexpr int REST = 0;
  static constexpr double THETA = 1.0 / 3.0;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <> struct Lattice<21> {
  static constexpr int Q = 21;
  static constexpr int R = 3;
  static constexpr int REST = 20;
  static constexpr double THETA = 2.0 / 3.0;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int t[21] = {1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, -2, -2, 2, 3, 0, -3, 0, 0};
    return t[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int t[21] = {0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 2, 2, -2, -2, 0, 3, 0, -3, 0};
    return t[i];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i < 4    ? 1.0 / 12.0
           : i < 8  ? 2.0 / 27.0
           : i < 12 ? 7.0 / 360.0
           : i < 16 ? 1.0 / 432.0
           : i < 20 ? 1.0 / 1620.0
                    : 91.0 / 324.0;
  }
};

// Device plane order of the populations: grouped by c_y (ascending), table
// order inside a group.  The populations of one group pull from the same
// source row, so their rows arrive in one TMA box of depth group_size.
template <int Q> struct Planes {
  using L = Lattice<Q>;
  struct Table {
    int plane[Q];  // plane of population i
  };
  static constexpr Table make() {
    Table t{};
    for (int i = 0; i < Q; ++i) {
      int p = 0;
      for (int j = 0; j < Q; ++j)
        if (L::cy(j) < L::cy(i) || (L::cy(j) == L::cy(i) && j < i)) ++p;
      t.plane[i] = p;
    }
    return t;
  }
  static constexpr Table kTable = make();
  // Use only in constant expressions (template arguments, constexpr locals).
  template <int I> static constexpr int plane = kTable.plane[I];
};

}  // namespace lbm
