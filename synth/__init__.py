"""Seeded synthetic workloads (signals, filters, states) shared by the tests,
the benchmark and the smoke check.  No filtering arithmetic lives here."""
