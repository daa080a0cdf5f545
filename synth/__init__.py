"""Seeded synthetic inputs (meshes, direction sets, materials) for the tests and the benchmark."""
